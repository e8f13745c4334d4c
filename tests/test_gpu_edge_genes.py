"""Edge genes on the GPU: fitness of G without the genes' edges and whole GA runs over edge ids,
bit-exact against the oracle."""
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
    from paper_2412_20980_gb300.gapa import GENES_EDGES

    b.build()
    c = Context(0)
    c.set_genes(GENES_EDGES)
    yield c
    torch.cuda.synchronize()
    c.close()


def _fit(ctx, g, pop):
    import torch

    ctx.graph_upload(g.row_ptr, g.col)
    out = ctx.fitness(torch.from_numpy(np.ascontiguousarray(pop, dtype=np.int32)).cuda())
    ctx.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("graph", ["ba", "hk", "path", "star", "grid"])
@pytest.mark.parametrize("objective", ["pc", "mcn"])
def test_edge_fitness_matches_oracle(ctx, graph, objective):
    from paper_2412_20980_gb300.gapa import OBJECTIVE_MCN, OBJECTIVE_PC

    g = {"ba": lambda: synth.ba_graph(3000, 3, 2), "hk": lambda: synth.hk_graph(2500, 3, 0.4, 3),
         "path": lambda: synth.named_graph("path", 5000), "star": lambda: synth.named_graph("star", 3000),
         "grid": lambda: synth.named_graph("grid", 3600)}[graph]()
    E = g.num_edges
    k = max(1, E // 8)
    rng = np.random.default_rng(E)
    pop = np.stack([rng.choice(E, k, replace=False) for _ in range(37)]).astype(np.int32)
    ctx.set_objective(OBJECTIVE_MCN if objective == "mcn" else OBJECTIVE_PC)
    try:
        got = _fit(ctx, g, pop)
    finally:
        ctx.set_objective(OBJECTIVE_PC)
    want = oracle.fitness(g.row_ptr, g.col, pop, "edges_mcn" if objective == "mcn" else "edges",
                          nthreads=oracle.max_threads())
    assert np.array_equal(got, want)


def test_edge_fitness_edge_cases(ctx):
    from paper_2412_20980_gb300 import GapaError

    star = synth.named_graph("star", 500)
    E = star.num_edges
    every = np.arange(E, dtype=np.int32)[None, :]
    assert _fit(ctx, star, every)[0] == 0  # nothing joined
    assert _fit(ctx, star, np.zeros((3, 0), np.int32)).tolist() == [500 * 499 // 2] * 3
    with pytest.raises(GapaError):  # an edge id outside [0, E) surfaces at sync
        _fit(ctx, star, np.array([[0, E]], np.int32))
    ctx.sync()


def test_edge_gene_run_bit_exact(ctx):
    g = synth.ba_graph(1200, 3, 7)
    ctx.graph_upload(g.row_ptr, g.col)
    from paper_2412_20980_gb300 import make_config

    cfg = make_config(k=200, pop=48, gens=15, tourn=2, pc=0.8, pm=0.05, seed=4)
    pop = ctx.pop_init(cfg)
    ctx.sync()
    assert np.array_equal(pop.cpu().numpy(), oracle.pop_init(g.num_edges, 200, 48, 4))
    got = ctx.run(cfg, want_pop=True)
    want = oracle.run(g.row_ptr, g.col, k=200, pop=48, gens=15, tourn=2, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr,
                      seed=4, flags=oracle.FLAG_EDGES, nthreads=oracle.max_threads())
    assert np.array_equal(got["traj"], want["traj"]) and got["best_fit"] == want["best_fit"]
    assert np.array_equal(got["best_set"], want["best_set"])
    assert np.array_equal(got["pop"].cpu().numpy(), want["pop"])


def test_edge_genes_limits(ctx):
    from paper_2412_20980_gb300 import Batch, Context, GapaError, Surrogate, make_config, make_surrogate_config
    from paper_2412_20980_gb300.gapa import GENES_EDGES

    big = synth.ba_graph(60000, 2, 1)  # labels alone exceed shared memory
    ctx.graph_upload(big.row_ptr, big.col)
    with pytest.raises(GapaError):
        ctx.fitness_host(np.zeros((2, 3), np.int32))
    small = synth.ba_graph(500, 2, 1)
    c2 = Context(0)
    c2.graph_upload(small.row_ptr, small.col)
    c2.set_genes(GENES_EDGES)
    with pytest.raises(GapaError):
        Batch([c2], [make_config(k=10, pop=8)])
    with pytest.raises(GapaError):
        Surrogate(c2, make_surrogate_config(batch=16, ring=64), seed=0)
    with pytest.raises(GapaError):  # k must stay below E
        c2.pop_init(make_config(k=small.num_edges, pop=4))
    c2.close()
