"""The forest-piece fitness kernel (GAPA_FITNESS_PIECE) inside the GA: whole runs replayed from
CUDA graphs, generations at the throughput workload's size, members deferred to the cut-local
kernel (hub-heavy sets, sets past the kernel's capacities) and the MCN objective, all equal to the
oracle bit-exactly (Section III-B loop, Section III-C fitness)."""
import numpy as np
import pytest

import oracle
import synth
from synth.graphs import disjoint_union

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2412_20980_gb300 import Context
    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import FITNESS_PIECE

    b.build()
    c = Context(0)
    c.set_fitness_kernel(FITNESS_PIECE)
    yield c
    torch.cuda.synchronize()
    c.close()


def _cfg(**kw):
    from paper_2412_20980_gb300 import make_config

    return make_config(**kw)


@pytest.mark.parametrize("make,k,s,gens", [
    (lambda: synth.ba_graph(5000, 3, 2), 250, 64, 30),
    (lambda: synth.hk_graph(8000, 4, 0.3, 3), 400, 96, 12),
    (lambda: synth.relabel(synth.ba_graph(6000, 2, 5), 4), 300, 50, 9),
])
def test_run_bit_exact(ctx, make, k, s, gens):
    g = make()
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=k, pop=s, gens=gens, tourn=2, pc=0.8, pm=0.02, seed=5)
    got = ctx.run(cfg, want_pop=True)
    want = oracle.run(g.row_ptr, g.col, k=k, pop=s, gens=gens, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                      seed=5, nthreads=oracle.max_threads())
    assert np.array_equal(got["traj"], want["traj"])
    assert np.array_equal(got["best_set"], want["best_set"])
    assert np.array_equal(got["pop"].cpu().numpy(), want["pop"])


@pytest.mark.parametrize("which", ["ba", "hk"])
def test_throughput_size_generations(ctx, which):
    """BA / HK n = 20000, k = 1000, population 1024: init, fitness and three generations."""
    g = synth.ba_graph(20000, 4, 1) if which == "ba" else synth.hk_graph(20000, 4, 0.3, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=1000, pop=1024, tourn=2, pc=0.8, pm=0.02, seed=0)
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    ctx.sync()
    wp = oracle.pop_init(g.n, 1000, 1024, 0)
    wf = oracle.fitness(g.row_ptr, g.col, wp, nthreads=oracle.max_threads())
    assert np.array_equal(fit.cpu().numpy(), wf)
    for gen in range(1, 4):
        pop, fit = ctx.generation(cfg, gen, pop, fit)
        ctx.sync()
        wp, wf = oracle.generation(g.row_ptr, g.col, wp, wf, gen, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                                   seed=0, nthreads=oracle.max_threads())
        assert np.array_equal(pop.cpu().numpy(), wp), gen
        assert np.array_equal(fit.cpu().numpy(), wf), gen


def test_deferred_members(ctx):
    """Members estimated to shatter the forests (many top hubs: deferred before any work) and
    members with more deletions than the kernel holds pieces for (deferred after trying), mixed
    with ordinary members in one launch."""
    import torch

    g = synth.hk_graph(20000, 4, 0.3, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(3)
    k = 6000
    rows = []
    for r in range(40):
        if r % 4 == 0:
            genes = np.concatenate([top[:3000], rng.choice(top[3000:], k - 3000, replace=False)])
        else:
            genes = rng.choice(g.n, k, replace=False)
        rows.append(genes)
    pop = np.stack(rows).astype(np.int32)
    got = ctx.fitness(torch.from_numpy(pop).cuda())
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads()))


def test_mcn_objective(ctx):
    import torch

    from paper_2412_20980_gb300.gapa import OBJECTIVE_MCN, OBJECTIVE_PC

    g = disjoint_union(synth.ba_graph(6000, 3, 1), synth.named_graph("path", 3000),
                       synth.ba_graph(4000, 2, 9))
    ctx.graph_upload(g.row_ptr, g.col)
    pop = synth.random_deletion_sets(g.n, 650, 48, 2)
    ctx.set_objective(OBJECTIVE_MCN)
    try:
        got = ctx.fitness(torch.from_numpy(pop).cuda())
        ctx.sync()
        assert np.array_equal(got.cpu().numpy(), oracle.fitness(g.row_ptr, g.col, pop, method="mcn"))
    finally:
        ctx.set_objective(OBJECTIVE_PC)
    got = ctx.fitness(torch.from_numpy(pop).cuda())
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.fitness(g.row_ptr, g.col, pop))
