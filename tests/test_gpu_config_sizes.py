"""Whole-trajectory parity at the workloads' own sizes.

The large workload (R-MAT scale 20, 2^24 edges, k = 10000, population 256) and the batched
workload (64 BA instances, n log-uniform in [500, 50000], populations 32..512) are run through
the C ABI for several generations - the Fig. 1 loop of Section III-B (Eqs. 2-11) with the exact
fitness of Section III-C - and every member, fitness value and best set is compared with the
oracle run on the host cores.  Integer results, so the bar is exact equality.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NT = None


def _nt():
    global NT
    if NT is None:
        NT = oracle.max_threads()
    return NT


@pytest.fixture(scope="module")
def rmat20():
    return synth.rmat_graph(20, 1 << 24, seed=1)


def _hub_heavy(g, k, s, seed):
    """Members holding many of the top hubs (what an evolved population holds), even rows
    more than odd rows, the rest drawn uniformly."""
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(seed)
    rows = []
    for r in range(s):
        h = (k // 2) if r % 2 == 0 else (k // 8)
        rest = rng.choice(top[h:], k - h, replace=False)
        rows.append(np.concatenate([top[:h], rest]))
    return np.stack(rows).astype(np.int32)


def test_large_rmat20_full_population_generations(rmat20):
    """R-MAT 2^20: pop_init, its fitness and three generations of all 256 members, each compared
    with the oracle member by member."""
    import torch

    from paper_2412_20980_gb300 import Context, make_config
    from paper_2412_20980_gb300 import build as b

    b.build()
    g = rmat20
    cfg = make_config(k=10000, pop=256, gens=3, tourn=2, pc=0.8, pm=0.02, seed=0)
    with Context(0) as ctx:
        ctx.graph_upload(g.row_ptr, g.col)
        pop = ctx.pop_init(cfg)
        fit = ctx.fitness(pop)
        ctx.sync()
        want_pop = oracle.pop_init(g.n, cfg.k, cfg.pop, cfg.seed)
        want_fit = oracle.fitness(g.row_ptr, g.col, want_pop, nthreads=_nt())
        assert np.array_equal(pop.cpu().numpy(), want_pop)
        assert np.array_equal(fit.cpu().numpy(), want_fit)
        for gen in range(1, 4):
            pop, fit = ctx.generation(cfg, gen, pop, fit)
            ctx.sync()
            want_pop, want_fit = oracle.generation(g.row_ptr, g.col, want_pop, want_fit, gen, tourn=2,
                                                   pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr, seed=cfg.seed,
                                                   nthreads=_nt())
            assert np.array_equal(pop.cpu().numpy(), want_pop), f"generation {gen}: population"
            assert np.array_equal(fit.cpu().numpy(), want_fit), f"generation {gen}: fitness"
        del torch


def test_large_rmat20_hub_heavy_generation(rmat20):
    """R-MAT 2^20 with a population whose members hold 625 to 5000 of the top hubs: the BFS tree
    shatters, so the interleaved-label path switches between neighbour sampling, the outside-node
    scan and the non-tree join.  Fitness of all 256 members and one generation from them."""
    import torch

    from paper_2412_20980_gb300 import Context, make_config
    from paper_2412_20980_gb300 import build as b

    b.build()
    g = rmat20
    cfg = make_config(k=10000, pop=256, gens=1, tourn=2, pc=0.8, pm=0.02, seed=5)
    pop_np = _hub_heavy(g, cfg.k, cfg.pop, 9)
    with Context(0) as ctx:
        ctx.graph_upload(g.row_ptr, g.col)
        pop = torch.from_numpy(pop_np).cuda()
        fit = ctx.fitness(pop)
        ctx.sync()
        want_fit = oracle.fitness(g.row_ptr, g.col, pop_np, nthreads=_nt())
        assert np.array_equal(fit.cpu().numpy(), want_fit)
        pop1, fit1 = ctx.generation(cfg, 1, pop, fit)
        ctx.sync()
        wp, wf = oracle.generation(g.row_ptr, g.col, pop_np, want_fit, 1, tourn=2, pc_thr=cfg.pc_thr,
                                   pm_thr=cfg.pm_thr, seed=cfg.seed, nthreads=_nt())
        assert np.array_equal(pop1.cpu().numpy(), wp)
        assert np.array_equal(fit1.cpu().numpy(), wf)


def _run_batch(specs, gens):
    from paper_2412_20980_gb300 import Batch, Context, make_config
    from paper_2412_20980_gb300 import build as b

    b.build()
    graphs, ctxs, cfgs = [], [], []
    for d in specs:
        g = synth.ba_graph(d["n"], d["m"], d["graph_seed"])
        c = Context(0)
        c.graph_upload(g.row_ptr, g.col)
        graphs.append(g)
        ctxs.append(c)
        cfgs.append(make_config(k=d["k"], pop=d["pop"], tourn=2, pc=0.8, pm=0.02, seed=d["index"]))
    bt = Batch(ctxs, cfgs)
    try:
        got = bt.run(gens)
    finally:
        bt.close()
        for c in ctxs:
            c.close()
    for i, (g, cfg) in enumerate(zip(graphs, cfgs)):
        want = oracle.run(g.row_ptr, g.col, k=cfg.k, pop=cfg.pop, gens=gens, tourn=cfg.tourn,
                          pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr, seed=cfg.seed, nthreads=_nt())
        assert np.array_equal(got["traj"][i], want["traj"]), (i, specs[i])
        assert got["best_fit"][i] == want["best_fit"], (i, specs[i])
        assert np.array_equal(got["best_sets"][i], want["best_set"]), (i, specs[i])


def test_batched_extremes_five_generations():
    """The batched workload's extremes in one batch for five generations: its largest instances
    (n = 33641 with population 512, n = 40722 with 256), its smallest (n = 517 with 32 and with
    512), and the top of its range, n = 50000 with m = 5 and population 512."""
    inst = {d["index"]: d for d in synth.batched_instances(64, seed=0)}
    specs = [inst[13], inst[50], inst[62], inst[56],
             {"index": 64, "n": 50000, "m": 5, "pop": 512, "k": 2500, "graph_seed": 65}]
    _run_batch(specs, 5)


def test_batched_workload_all_instances():
    """All 64 instances of the batched workload in one batch, three generations, each instance
    against its own oracle run."""
    _run_batch(synth.batched_instances(64, seed=0), 3)
