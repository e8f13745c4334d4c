"""GPU fitness parity: libgapa.so's batched pairwise connectivity equals the oracle bit-exactly.

Fitness is integer (int64), so the bar is exact equality, element by element.
Covers hand-worked values, exhaustive subsets of tiny graphs, the benchmark
graphs (BA/HK n = 20000, k = 1000, s = 1024), graphs too large for shared
memory (global labels and the sparse kernel, which every test also runs on
small graphs), and degenerate sets and graphs.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pc_worked_examples.json")


@pytest.fixture(scope="module", params=["sparse", "piece", "tree_local", "tree", "tree_join", "tree_scan", "sampled",
                                        "edges"])
def ctx(request):
    import torch

    from paper_2412_20980_gb300 import Context
    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import (FITNESS_EDGES, FITNESS_PIECE, FITNESS_SAMPLED, FITNESS_SPARSE,
                                             FITNESS_TREE, FITNESS_TREE_JOIN, FITNESS_TREE_LOCAL, FITNESS_TREE_SCAN)

    b.build()
    c = Context(0)
    c.set_fitness_kernel({"tree": FITNESS_TREE, "tree_join": FITNESS_TREE_JOIN, "tree_scan": FITNESS_TREE_SCAN,
                          "tree_local": FITNESS_TREE_LOCAL, "piece": FITNESS_PIECE, "sampled": FITNESS_SAMPLED,
                          "edges": FITNESS_EDGES, "sparse": FITNESS_SPARSE}[request.param])
    c.variant_name = request.param
    yield c
    torch.cuda.synchronize()
    c.close()


def gpu_fit(ctx, g, pop):
    import torch

    ctx.graph_upload(g.row_ptr, g.col)
    p = torch.from_numpy(np.ascontiguousarray(pop, dtype=np.int32)).cuda()
    f = ctx.fitness(p)
    ctx.sync()
    return f.cpu().numpy()


def test_worked_examples(ctx):
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        e = np.array(case["edges"], dtype=np.int64).reshape(-1, 2)
        g = synth.csr_from_edges(case["n"], e[:, 0], e[:, 1])
        for s in case["sets"]:
            got = gpu_fit(ctx, g, np.array([s["del"]], dtype=np.int32).reshape(1, -1))
            assert got[0] == s["pc"], (case["name"], s)


@pytest.mark.parametrize("seed,n,m", [(1, 12, 16), (3, 11, 25), (5, 10, 9)])
def test_exhaustive_subsets(ctx, seed, n, m):
    g = synth.er_graph(n, m, seed)
    for k in range(n + 1):
        combos = list(itertools.combinations(range(n), k))
        pop = np.array(combos, dtype=np.int32).reshape(len(combos), k)
        assert np.array_equal(gpu_fit(ctx, g, pop), oracle.fitness(g.row_ptr, g.col, pop)), k


@pytest.mark.parametrize("make", [
    lambda: synth.ba_graph(20000, 4, 1),
    lambda: synth.hk_graph(20000, 4, 0.3, 1),
])
def test_benchmark_graphs_full_population(ctx, make):
    g = make()
    pop = synth.random_deletion_sets(g.n, 1000, 1024, 0)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


@pytest.mark.parametrize("graph", ["ba", "hk"])
@pytest.mark.parametrize("hubs", [0, 100, 500, 1000])
def test_benchmark_graphs_hub_heavy(ctx, graph, hubs):
    """Deletion sets holding the top hubs of the benchmark graphs (what an evolved population
    deletes): the BFS tree shatters, the list of nodes outside the first live node's piece grows
    from a few hundred to most of the graph, and the cut-local kernel moves from its list to the
    full pipeline; 33 members (a ragged last warp of genes), odd rows with half the hubs."""
    g = synth.ba_graph(20000, 4, 1) if graph == "ba" else synth.hk_graph(20000, 4, 0.3, 1)
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(hubs + 7)
    rows = []
    for r in range(33):
        h = hubs if r % 2 == 0 else hubs // 2
        rest = rng.choice(top[h:], 1000 - h, replace=False)
        rows.append(rng.permutation(np.concatenate([top[:h], rest])))
    pop = np.stack(rows).astype(np.int32)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


@pytest.mark.parametrize("make,k,s", [
    (lambda: synth.ba_graph(1000, 3, 1), 50, 100),
    (lambda: synth.relabel(synth.ba_graph(5000, 2, 4), 9), 500, 64),
    (lambda: synth.rmat_graph(12, 30000, seed=3, chunk=1 << 15), 200, 48),
    (lambda: synth.named_graph("grid", 40000), 4000, 16),
])
def test_various_graphs(ctx, make, k, s):
    g = make()
    pop = synth.random_deletion_sets(g.n, k, s, 1)
    assert np.array_equal(gpu_fit(ctx, g, pop), oracle.fitness(g.row_ptr, g.col, pop))


@pytest.mark.parametrize("n,k", [(100000, 2000), (60000, 3000)])
def test_global_label_path(ctx, n, k):
    """Too many labels for shared memory (n = 100000: 400 KB; n = 60000 sits between the
    shared-memory limit and 2^16): the global-memory variant."""
    g = synth.ba_graph(n, 3, 1)
    pop = synth.random_deletion_sets(g.n, k, 40, 2)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


def test_global_label_partial_group(ctx):
    """37 members: the last interleaved group of eight is partial."""
    g = synth.relabel(synth.hk_graph(70000, 3, 0.3, 5), 3)
    pop = synth.random_deletion_sets(g.n, 3500, 37, 9)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


def test_full_size_rmat_sampled_members(ctx):
    """R-MAT scale 20 with 2^24 edges, k = 10000, s = 256 (the large configuration, evaluated as
    one batch); eight members spread over the batch are checked against the oracle one by one."""
    if ctx.variant_name not in ("tree", "sparse"):
        pytest.skip("full-size check runs on the two large-graph kernels only")
    g = synth.rmat_graph(20, 1 << 24, seed=1)
    pop = synth.random_deletion_sets(g.n, 10000, 256, 0)
    got = gpu_fit(ctx, g, pop)
    rows = [0, 7, 8, 100, 127, 128, 200, 255]
    want = oracle.fitness(g.row_ptr, g.col, pop[rows], nthreads=oracle.max_threads())
    assert np.array_equal(got[rows], want)
    # properties at any size: PC <= C(n-k, 2); and a hub-heavy member reduces PC
    n, k = g.n, 10000
    assert np.all(got <= (n - k) * (n - k - 1) // 2)


def test_global_label_path_rmat(ctx):
    g = synth.rmat_graph(17, 1 << 20, seed=1, chunk=1 << 20)
    pop = synth.random_deletion_sets(g.n, 1300, 24, 5)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


@pytest.mark.parametrize("hubs", [0, 20, 200, 1300])
def test_global_label_path_hub_heavy(ctx, hubs):
    """A dense R-MAT graph (8 edges per node, so the sampling / giant / scan steps run) whose
    deletion sets hold the top hubs: the BFS tree shatters and the groups move between the
    outside-node scan and the non-tree join; sizes 17 members, a group and a ragged tail."""
    if ctx.variant_name not in ("tree", "sparse"):
        pytest.skip("runs on the two large-graph kernels only")
    g = synth.rmat_graph(17, 1 << 20, seed=3, chunk=1 << 20)
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(hubs)
    rows = []
    for r in range(17):
        h = min(hubs, 1300) if r % 2 == 0 else hubs // 2
        rest = rng.choice(top[h:], 1300 - h, replace=False)
        rows.append(np.concatenate([top[:h], rest]))
    pop = np.stack(rows).astype(np.int32)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


@pytest.mark.parametrize("graph", ["rmat", "ba"])
def test_top_hub_combinations(ctx, graph):
    """Members deleting neither, the first, the second or both of the two highest-degree nodes, with
    and without more hubs: the sparse kernel evaluates each on the forest of G without the deleted
    top hubs' edges (every routing case), the other kernels on G; all equal the oracle."""
    g = (synth.rmat_graph(17, 1 << 20, seed=4, chunk=1 << 20) if graph == "rmat"
         else synth.ba_graph(30000, 3, 5))
    top = np.argsort(-g.degrees(), kind="stable")
    k = 600
    rng = np.random.default_rng(19)
    heads = [[], [0], [1], [0, 1], [1, 2, 3], [0, 2, 3, 4], [0, 1, 2, 3, 4, 5, 6, 7]]
    rows = []
    for h in heads:
        for _ in range(3):
            fixed = top[h].astype(np.int64)
            rest = rng.choice(top[8:], k - len(fixed), replace=False)
            rows.append(rng.permutation(np.concatenate([fixed, rest])))
    pop = np.stack(rows).astype(np.int32)
    want = oracle.fitness(g.row_ptr, g.col, pop, nthreads=oracle.max_threads())
    assert np.array_equal(gpu_fit(ctx, g, pop), want)


def test_adversarial_graphs(ctx):
    path = synth.named_graph("path", 30000)  # deep union-find chains
    pop = np.zeros((1, 0), dtype=np.int32)
    assert gpu_fit(ctx, path, pop)[0] == 30000 * 29999 // 2
    pop = synth.random_deletion_sets(path.n, 100, 8, 3)
    assert np.array_equal(gpu_fit(ctx, path, pop), oracle.fitness(path.row_ptr, path.col, pop))
    star = synth.named_graph("star", 20001)  # one hot root
    pop = np.array([[0], [1], [20000]], dtype=np.int32)
    assert list(gpu_fit(ctx, star, pop)) == [0, 20000 * 19999 // 2, 20000 * 19999 // 2]
    empty = synth.named_graph("empty", 5000)  # all isolated
    assert gpu_fit(ctx, empty, np.zeros((3, 0), dtype=np.int32)).tolist() == [0, 0, 0]
    # all neighbours of the hub deleted
    ba = synth.ba_graph(3000, 2, 7)
    hub = int(np.argmax(ba.degrees()))
    nb = ba.col[ba.row_ptr[hub]:ba.row_ptr[hub + 1]]
    pop = nb.reshape(1, -1).astype(np.int32)
    assert np.array_equal(gpu_fit(ctx, ba, pop), oracle.fitness(ba.row_ptr, ba.col, pop))


def test_degenerate_sets(ctx):
    g = synth.ba_graph(2000, 3, 2)
    n = g.n
    # k = 0, k = n - 1, k = n, repeated genes
    assert gpu_fit(ctx, g, np.zeros((2, 0), dtype=np.int32)).tolist() == [n * (n - 1) // 2] * 2
    allbut = np.arange(1, n, dtype=np.int32).reshape(1, -1)
    assert gpu_fit(ctx, g, allbut).tolist() == [0]
    assert gpu_fit(ctx, g, np.arange(n, dtype=np.int32).reshape(1, -1)).tolist() == [0]
    rep = np.array([[5, 5, 5, 9], [9, 5, 9, 5]], dtype=np.int32)
    want = oracle.fitness(g.row_ptr, g.col, rep)
    assert np.array_equal(gpu_fit(ctx, g, rep), want) and want[0] == want[1]


def test_empty_population(ctx):
    import torch

    g = synth.ba_graph(500, 2, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    f = ctx.fitness(torch.zeros((0, 10), dtype=torch.int32, device="cuda"))
    ctx.sync()
    assert f.numel() == 0


def test_bad_gene_reported_at_sync(ctx):
    import torch

    from paper_2412_20980_gb300 import GapaError

    g = synth.ba_graph(500, 2, 1)
    ctx.graph_upload(g.row_ptr, g.col)
    pop = torch.tensor([[1, 2, 500]], dtype=torch.int32, device="cuda")
    ctx.fitness(pop)
    with pytest.raises(GapaError) as ei:
        ctx.sync()
    assert ei.value.code == -7
    # the context stays usable
    ok = ctx.fitness(torch.tensor([[1, 2, 3]], dtype=torch.int32, device="cuda"))
    ctx.sync()
    assert ok.item() == oracle.fitness(g.row_ptr, g.col, np.array([[1, 2, 3]]))[0]


def test_host_entry_point_matches_device(ctx):
    g = synth.hk_graph(3000, 3, 0.3, 4)
    pop = synth.random_deletion_sets(g.n, 150, 33, 8)
    ctx.graph_upload(g.row_ptr, g.col)
    host = ctx.fitness_host(pop)
    assert np.array_equal(host, gpu_fit(ctx, g, pop))
    assert np.array_equal(host, oracle.fitness(g.row_ptr, g.col, pop))


def test_invalid_graphs_rejected(ctx):
    from paper_2412_20980_gb300 import GapaError

    rp = np.array([0, 1, 2], dtype=np.int32)
    for col, code in [(np.array([1, 1], dtype=np.int32), -2),  # fine shape but... 0->1, 1->1 self loop
                      (np.array([0, 0], dtype=np.int32), -2),
                      (np.array([1, 5], dtype=np.int32), -2)]:
        with pytest.raises(GapaError) as ei:
            ctx.graph_upload(rp, col)
        assert ei.value.code == code
    # asymmetric: 0->1, 1->2, 2->? (row 2 empty)
    with pytest.raises(GapaError):
        ctx.graph_upload(np.array([0, 1, 2, 2], dtype=np.int32), np.array([1, 2], dtype=np.int32))
    # repeated arc
    with pytest.raises(GapaError):
        ctx.graph_upload(np.array([0, 2, 4], dtype=np.int32), np.array([1, 1, 0, 0], dtype=np.int32))


@pytest.mark.parametrize("graph", ["ba", "path", "star", "hub_deleted", "large"])
def test_mcn_objective_matches_oracle(ctx, graph):
    """The maximum connectivity number objective, on the shared-memory and the global-label paths."""
    from paper_2412_20980_gb300.gapa import OBJECTIVE_MCN, OBJECTIVE_PC

    if graph == "large" and ctx.variant_name not in ("tree", "sparse"):
        pytest.skip("runs on the two large-graph kernels only")
    g = {"ba": lambda: synth.ba_graph(3000, 2, 4), "path": lambda: synth.named_graph("path", 4000),
         "star": lambda: synth.named_graph("star", 2500), "hub_deleted": lambda: synth.ba_graph(2000, 1, 6),
         "large": lambda: synth.ba_graph(100000, 3, 2)}[graph]()
    k = max(1, g.n // 20)
    pop = synth.random_deletion_sets(g.n, k, 40, 11)
    if graph in ("star", "hub_deleted"):
        hubs = np.argsort(-g.degrees(), kind="stable")[:k].astype(np.int32)
        pop[0] = hubs  # the centre / the hubs: many small components
    ctx.set_objective(OBJECTIVE_MCN)
    try:
        got = gpu_fit(ctx, g, pop)
    finally:
        ctx.set_objective(OBJECTIVE_PC)
    want = oracle.fitness(g.row_ptr, g.col, pop, "mcn", nthreads=oracle.max_threads())
    assert np.array_equal(got, want)
