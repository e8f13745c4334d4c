"""Batched runs: every instance of a batch equals the oracle's run of that instance bit-exactly."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SPECS = [  # (n, m, pop, seed): uneven sizes and populations
    (300, 2, 8, 11),
    (800, 3, 16, 12),
    (1500, 2, 32, 13),
    (3000, 4, 64, 14),
    (6000, 3, 24, 15),
    (12000, 2, 40, 16),
]


def _batch(specs, teams=None, variant=None):
    from paper_2412_20980_gb300 import Batch, Context, make_config
    from paper_2412_20980_gb300 import build as b

    b.build()
    graphs, ctxs, cfgs = [], [], []
    for (n, m, pop, seed) in specs:
        g = synth.ba_graph(n, m, seed)
        c = Context(0)
        if variant is not None:
            c.set_fitness_kernel(variant)
        c.graph_upload(g.row_ptr, g.col)
        graphs.append(g)
        ctxs.append(c)
        cfgs.append(make_config(k=max(1, round(0.05 * n)), pop=pop, tourn=2, pc=0.8, pm=0.02, seed=seed))
    bt = Batch(ctxs, cfgs)
    if teams is not None:
        bt.teams = teams
    return bt, graphs, ctxs, cfgs


def _oracle(g, cfg, gens):
    return oracle.run(g.row_ptr, g.col, k=cfg.k, pop=cfg.pop, gens=gens, tourn=cfg.tourn, pc_thr=cfg.pc_thr,
                      pm_thr=cfg.pm_thr, seed=cfg.seed, nthreads=oracle.max_threads())


@pytest.mark.parametrize("gens", [0, 1, 7, 10])
def test_batch_matches_oracle_per_instance(gens):
    bt, graphs, ctxs, cfgs = _batch(SPECS)
    got = bt.run(gens)
    for i, (g, cfg) in enumerate(zip(graphs, cfgs)):
        want = _oracle(g, cfg, gens)
        assert np.array_equal(got["traj"][i], want["traj"]), i
        assert got["best_fit"][i] == want["best_fit"], i
        assert np.array_equal(got["best_sets"][i], want["best_set"]), i
    bt.close()


@pytest.mark.parametrize("teams", [[1] * 6, [8, 8, 4, 4, 2, 1], [2, 4, 8, 2, 1, 1]])
def test_batch_cut_local_kernel_matches_oracle(teams):
    """Contexts set to the cut-local kernel: every team count runs tree16_member_local in its
    slice of the persistent kernel (bulk copy and mbarrier reused member after member)."""
    from paper_2412_20980_gb300.gapa import FITNESS_TREE_LOCAL

    bt, graphs, ctxs, cfgs = _batch(SPECS, teams=teams, variant=FITNESS_TREE_LOCAL)
    got = bt.run(7)
    for i, (g, cfg) in enumerate(zip(graphs, cfgs)):
        want = _oracle(g, cfg, 7)
        assert np.array_equal(got["traj"][i], want["traj"]), i
        assert np.array_equal(got["best_sets"][i], want["best_set"]), i
    bt.close()


def test_team_counts_do_not_change_results():
    bt, graphs, ctxs, cfgs = _batch(SPECS, teams=[1] * len(SPECS))
    a = bt.run(6)
    bt.teams = [8, 8, 4, 2, 1, 1]
    b = bt.run(6)
    assert np.array_equal(a["traj"], b["traj"]) and np.array_equal(a["best_fit"], b["best_fit"])
    bt.close()


def test_autotune_writes_and_reuses_cache(tmp_path):
    cache = str(tmp_path / "teams.json")
    bt, graphs, ctxs, cfgs = _batch(SPECS)
    before = bt.run(4)
    bt.autotune(cache)
    chosen = bt.teams
    assert all(t in (1, 2, 4, 8) for t in chosen)
    data = json.load(open(cache))
    assert len(data) == 1 and len(next(iter(data.values()))) >= 1
    after = bt.run(4)
    assert np.array_equal(before["traj"], after["traj"])
    bt.close()
    bt2, *_ = _batch(SPECS)
    bt2.autotune(cache)  # served from the cache
    assert bt2.teams == chosen
    bt2.close()


def test_batch_equals_single_runs():
    from paper_2412_20980_gb300 import make_config

    bt, graphs, ctxs, cfgs = _batch(SPECS[:3])
    got = bt.run(9)
    for i, (c, cfg) in enumerate(zip(ctxs, cfgs)):
        cfg1 = make_config(k=cfg.k, pop=cfg.pop, gens=9, seed=cfg.seed)
        single = c.run(cfg1)
        assert np.array_equal(single["traj"], got["traj"][i])
    bt.close()


def test_batch_rejects_large_graph():
    from paper_2412_20980_gb300 import Batch, Context, GapaError, make_config

    g = synth.ba_graph(100000, 2, 1)
    c = Context(0)
    c.graph_upload(g.row_ptr, g.col)
    with pytest.raises(GapaError) as ei:
        Batch([c], [make_config(k=100, pop=8)])
    assert ei.value.code == -1
