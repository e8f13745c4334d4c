"""GPU genetic-operator parity: populations, fitness and whole trajectories equal the oracle bit-exactly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2412_20980_gb300 import Context
    from paper_2412_20980_gb300 import build as b

    b.build()
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _cfg(**kw):
    from paper_2412_20980_gb300 import make_config

    return make_config(**kw)


@pytest.mark.parametrize("n,k,s,seed", [(1000, 50, 100, 0), (20000, 1000, 64, 7), (12, 11, 40, 3),
                                         (40, 39, 17, 5), (300, 0, 5, 1), (100000, 2000, 8, 2)])
def test_pop_init_bit_exact(ctx, n, k, s, seed):
    g = synth.named_graph("path", n)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=k, pop=s, seed=seed)
    pop = ctx.pop_init(cfg)
    ctx.sync()
    assert np.array_equal(pop.cpu().numpy(), oracle.pop_init(n, k, s, seed))


def _gen_case(ctx, g, k, s, pc, pm, tourn, seed, flags, gens, lam=0):
    import torch

    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=k, pop=s, tourn=tourn, pc=pc, pm=pm, seed=seed, flags=flags, lam=lam)
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    wp = oracle.pop_init(g.n, k, s, seed)
    wf = oracle.fitness(g.row_ptr, g.col, wp)
    for gen in range(1, gens + 1):
        pop, fit = ctx.generation(cfg, gen, pop, fit)
        wp, wf = oracle.generation(g.row_ptr, g.col, wp, wf, gen, tourn=tourn, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                                   seed=seed, flags=flags, lam=lam, nthreads=oracle.max_threads())
        ctx.sync()
        assert np.array_equal(pop.cpu().numpy(), wp), gen
        assert np.array_equal(fit.cpu().numpy(), wf), gen


@pytest.mark.parametrize("pc,pm,tourn,flags", [(0.8, 0.02, 2, 0), (0.0, 0.0, 2, 0), (1.0, 0.0, 3, 0),
                                                (0.5, 0.3, 2, 0), (0.8, 0.02, 2, 1), (0.6, 0.2, 1, 0)])
def test_generation_bit_exact_c0_graph(ctx, pc, pm, tourn, flags):
    _gen_case(ctx, synth.ba_graph(1000, 3, 1), 50, 100, pc, pm, tourn, 0, flags, 4)


def test_generation_heavy_duplicates(ctx):
    _gen_case(ctx, synth.named_graph("cycle", 14), 12, 30, 0.5, 0.5, 2, 11, 0, 12)
    _gen_case(ctx, synth.er_graph(60, 90, 2), 55, 24, 0.7, 0.9, 2, 12, 0, 6)


def test_generation_c1_sizes(ctx):
    _gen_case(ctx, synth.hk_graph(20000, 4, 0.3, 1), 1000, 128, 0.8, 0.02, 2, 0, 0, 2)


def test_generation_large_graph(ctx):
    _gen_case(ctx, synth.ba_graph(100000, 3, 1), 2000, 16, 0.8, 0.02, 2, 4, 0, 2)


@pytest.mark.parametrize("gens", [0, 1, 2, 5, 100])
def test_run_bit_exact_c0(ctx, gens):
    g = synth.ba_graph(1000, 3, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=50, pop=100, gens=gens, tourn=2, pc=0.8, pm=0.02, seed=0)
    got = ctx.run(cfg, want_pop=True)
    want = oracle.run(g.row_ptr, g.col, k=50, pop=100, gens=gens, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                      seed=0)
    assert np.array_equal(got["traj"], want["traj"])
    assert got["best_fit"] == want["best_fit"]
    assert np.array_equal(got["best_set"], want["best_set"])
    assert np.array_equal(got["pop"].cpu().numpy(), want["pop"])


def test_run_repeatable_and_matches_stepwise(ctx):
    import torch

    g = synth.hk_graph(2000, 3, 0.3, 2)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=100, pop=64, gens=9, seed=123)
    a = ctx.run(cfg, want_pop=True)
    b = ctx.run(cfg, want_pop=True)
    assert np.array_equal(a["traj"], b["traj"]) and torch.equal(a["pop"], b["pop"])
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    for gen in range(1, 10):
        pop, fit = ctx.generation(cfg, gen, pop, fit)
    ctx.sync()
    assert torch.equal(pop, a["pop"])


def test_generation_host_matches_device(ctx):
    g = synth.ba_graph(1500, 2, 3)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=75, pop=50, seed=9)
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    p1, f1 = ctx.generation(cfg, 1, pop, fit)
    ctx.sync()
    hp, hf = ctx.generation_host(cfg, 1, pop.cpu().numpy(), fit.cpu().numpy())
    assert np.array_equal(hp, p1.cpu().numpy()) and np.array_equal(hf, f1.cpu().numpy())


def test_invalid_configs(ctx):
    from paper_2412_20980_gb300 import GapaError

    g = synth.ba_graph(500, 2, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    for kw in (dict(k=500, pop=10), dict(k=5, pop=1), dict(k=5, pop=10, tourn=0), dict(k=5, pop=10, elite=2),
               dict(k=-1, pop=10), dict(k=5, pop=10, flags=8)):
        import torch

        out = torch.empty((16, 8), dtype=torch.int32, device="cuda")  # never written: the call is rejected first
        with pytest.raises(GapaError) as ei:
            ctx.pop_init(_cfg(**kw), out=out)
        assert ei.value.code == -1


ROULETTE, MPL = 4, 2


@pytest.mark.parametrize("flags,lam,pm", [(ROULETTE, 0, 0.02), (MPL, 150, 0.02), (MPL | ROULETTE, 64, 0.1),
                                          (MPL, 1, 0.02), (MPL, 400, 0.3)])
def test_selection_and_elitism_variants_bit_exact(ctx, flags, lam, pm):
    """Roulette (Eq. 5) and (mu+lambda) truncation (Eqs. 10-11) against the oracle."""
    _gen_case(ctx, synth.ba_graph(1000, 3, 1), 50, 100, 0.8, pm, 2, 3, flags, 4, lam=lam)


def test_mu_plus_lambda_large_graph(ctx):
    _gen_case(ctx, synth.ba_graph(100000, 3, 1), 2000, 16, 0.8, 0.02, 2, 4, MPL | ROULETTE, 2, lam=40)


@pytest.mark.parametrize("gens", [1, 6])
def test_run_variants_bit_exact(ctx, gens):
    g = synth.hk_graph(3000, 3, 0.3, 6)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=150, pop=64, gens=gens, tourn=2, pc=0.8, pm=0.05, seed=8, flags=MPL | ROULETTE, lam=192)
    got = ctx.run(cfg, want_pop=True)
    want = oracle.run(g.row_ptr, g.col, k=150, pop=64, gens=gens, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                      seed=8, flags=MPL | ROULETTE, lam=192, nthreads=oracle.max_threads())
    assert np.array_equal(got["traj"], want["traj"])
    assert np.array_equal(got["pop"].cpu().numpy(), want["pop"])
    assert np.array_equal(got["best_set"], want["best_set"])


def test_variant_configs_rejected(ctx):
    import torch

    from paper_2412_20980_gb300 import GapaError

    g = synth.ba_graph(500, 2, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    out = torch.empty((16, 8), dtype=torch.int32, device="cuda")
    for kw in (dict(k=5, pop=10, flags=MPL, lam=0), dict(k=5, pop=10, flags=MPL | 1, lam=5),
               dict(k=5, pop=10000, flags=MPL, lam=7000)):
        with pytest.raises(GapaError):
            ctx.pop_init(_cfg(**kw), out=out)


@pytest.mark.parametrize("flags", [0, 4])
def test_offspring_plus_sliced_fitness_equals_generation(ctx, flags):
    """The member split of one population: operators once, fitness by slices (two simulated ranks)."""
    import torch

    from paper_2412_20980_gb300 import GapaError
    from paper_2412_20980_gb300 import dist as gd

    g = synth.ba_graph(3000, 3, 5)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=150, pop=77, tourn=2, pc=0.8, pm=0.03, seed=4, flags=flags)
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    want_p, want_f = ctx.generation(cfg, 3, pop, fit)
    p2, f2 = torch.empty_like(pop), torch.full_like(fit, -7)
    ctx.offspring(cfg, 3, pop, fit, p2, f2)
    for r in range(2):
        lo, hi = gd.shard_bounds(cfg.pop - 1, 2, r)
        ctx.fitness(p2[1 + lo:1 + hi], out=f2[1 + lo:1 + hi])
    ctx.sync()
    assert torch.equal(p2, want_p) and torch.equal(f2, want_f)
    with pytest.raises(GapaError):
        ctx.offspring(_cfg(k=150, pop=77, seed=4, flags=2, lam=64), 3, pop, fit, p2, f2)


def test_mcn_run_bit_exact(ctx):
    """A whole run under the MCN objective follows the oracle's MCN run."""
    from paper_2412_20980_gb300.gapa import OBJECTIVE_MCN, OBJECTIVE_PC

    g = synth.ba_graph(1500, 2, 9)
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = _cfg(k=75, pop=64, gens=20, tourn=2, pc=0.8, pm=0.02, seed=6)
    ctx.set_objective(OBJECTIVE_MCN)
    try:
        got = ctx.run(cfg, want_pop=True)
    finally:
        ctx.set_objective(OBJECTIVE_PC)
    want = oracle.run(g.row_ptr, g.col, k=75, pop=64, gens=20, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                      seed=6, flags=oracle.FLAG_MCN, nthreads=oracle.max_threads())
    assert np.array_equal(got["traj"], want["traj"]) and got["best_fit"] == want["best_fit"]
    assert np.array_equal(got["best_set"], want["best_set"])
    assert np.array_equal(got["pop"].cpu().numpy(), want["pop"])
