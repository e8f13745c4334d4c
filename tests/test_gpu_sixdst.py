"""The SixDST dense reachability objectives (Eqs. 14-17) on the tensor cores against the dense
reference; exact 0/1 products, so the comparison is bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from oracle import sixdst_ref as sx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["tma", "mma_sync", "tcgen05", "tcgen05_128"])
def ctx(request):
    import torch

    from paper_2412_20980_gb300 import Context
    from paper_2412_20980_gb300 import build as b

    b.build()
    c = Context(0)
    # tcgen05 and tma: 256-wide tiles where the padded size is a multiple of 256 (n = 150, 200, 500,
    # 700 below; tma loads them by TMA with split producer and product roles), 128-wide otherwise;
    # tcgen05_128: 128-wide tiles throughout
    c.set_sixdst_kernel({"mma_sync": 0, "tcgen05": 1, "tcgen05_128": 2, "tma": 3}[request.param])
    yield c
    torch.cuda.synchronize()
    c.close()


def _fit(ctx, g, pop, hops, objective):
    import torch

    from paper_2412_20980_gb300.gapa import OBJECTIVE_PC, OBJECTIVE_SIXDST_MCN, OBJECTIVE_SIXDST_PC

    ctx.graph_upload(g.row_ptr, g.col)
    ctx.set_objective(OBJECTIVE_SIXDST_MCN if objective == "mcn" else OBJECTIVE_SIXDST_PC)
    ctx.set_sixdst_hops(hops)
    try:
        out = ctx.fitness(torch.from_numpy(np.ascontiguousarray(pop, dtype=np.int32)).cuda())
        ctx.sync()
    finally:
        ctx.set_objective(OBJECTIVE_PC)
        ctx.set_sixdst_hops(6)
    return out.cpu().numpy()


@pytest.mark.parametrize("graph", ["ba", "er", "path", "star", "ragged"])
@pytest.mark.parametrize("hops", [1, 2, 3, 6])
@pytest.mark.parametrize("objective", ["pc", "mcn"])
def test_sixdst_matches_dense_reference(ctx, graph, hops, objective):
    g = {"ba": lambda: synth.ba_graph(300, 2, 1), "er": lambda: synth.er_graph(500, 900, 2),
         "path": lambda: synth.named_graph("path", 200), "star": lambda: synth.named_graph("star", 150),
         "ragged": lambda: synth.hk_graph(77, 2, 0.3, 5)}[graph]()
    k = max(1, g.n // 10)
    pop = synth.random_deletion_sets(g.n, k, 19, hops)
    if graph == "star":
        pop[0, 0] = 0 if 0 not in pop[0] else pop[0, 0]  # the centre in one member
    want = sx.fitness(g.row_ptr, g.col, pop, hops=hops, objective=objective)
    assert np.array_equal(_fit(ctx, g, pop, hops, objective), want)


def test_sixdst_reaches_exact_objectives(ctx):
    g = synth.ba_graph(700, 2, 3)
    pop = synth.random_deletion_sets(g.n, 60, 33, 4)
    assert np.array_equal(_fit(ctx, g, pop, 700, "pc"), oracle.fitness(g.row_ptr, g.col, pop))
    assert np.array_equal(_fit(ctx, g, pop, 700, "mcn"), oracle.fitness(g.row_ptr, g.col, pop, "mcn"))


def test_sixdst_run_and_limits(ctx):
    import torch

    from paper_2412_20980_gb300 import Batch, GapaError, make_config
    from paper_2412_20980_gb300.gapa import OBJECTIVE_PC, OBJECTIVE_SIXDST_PC

    g = synth.ba_graph(500, 1, 2)  # a tree, as the paper's BA500
    ctx.graph_upload(g.row_ptr, g.col)
    cfg = make_config(k=50, pop=40, gens=8, tourn=2, pc=0.5, pm=0.3, seed=1)
    ctx.set_objective(OBJECTIVE_SIXDST_PC)
    try:
        res = ctx.run(cfg, want_pop=True)
        with pytest.raises(GapaError):
            Batch([ctx], [cfg])
    finally:
        ctx.set_objective(OBJECTIVE_PC)
    assert np.all(np.diff(res["traj"]) <= 0)
    assert res["best_fit"] == sx.sixdst_fitness(g.row_ptr, g.col, res["best_set"], hops=6)
    assert res["pop"].cpu().numpy().max() < g.n
    big = synth.ba_graph(9000, 2, 1)
    ctx.graph_upload(big.row_ptr, big.col)
    ctx.set_objective(OBJECTIVE_SIXDST_PC)
    try:
        with pytest.raises(GapaError):
            ctx.fitness(torch.zeros((2, 3), dtype=torch.int32, device="cuda"))
    finally:
        ctx.set_objective(OBJECTIVE_PC)


def test_bounded_wait_times_out_and_context_survives(ctx):
    """The device-side wait of the tcgen05 products on a barrier that nothing completes runs out,
    is reported as a timeout, and the context keeps working."""
    from paper_2412_20980_gb300.gapa import OBJECTIVE_PC

    assert ctx.selftest_wait(1 << 12) == -5  # GAPA_ERR_TIMEOUT
    g = synth.ba_graph(400, 2, 8)
    ctx.graph_upload(g.row_ptr, g.col)
    ctx.set_objective(OBJECTIVE_PC)
    pop = synth.random_deletion_sets(g.n, 20, 4, 1)
    assert np.array_equal(ctx.fitness_host(pop), oracle.fitness(g.row_ptr, g.col, pop))


def test_read_bandwidth_probe(ctx):
    """The bandwidth probe the bench uses for its L2 denominator: a buffer inside L2 reads faster
    than one far above it, and both figures are physically plausible for one GPU."""
    from paper_2412_20980_gb300 import GapaError

    l2 = ctx.read_bandwidth(64 << 20, 5)
    hbm = ctx.read_bandwidth(1 << 30, 3)
    assert 500.0 < hbm < 20000.0 and l2 > hbm, (l2, hbm)
    with pytest.raises(GapaError):
        ctx.read_bandwidth(1000, 1)  # not a multiple of 16 and below 1 MiB
