"""Pins of the oracle's fitness (pairwise connectivity of the residual graph).

PC(D) = sum over components C of G[V \\ D] of |C|(|C|-1)/2; node deletion removes
every incident edge (Section III-C, Eq. 13); PC(G) is the CND quality metric of
the paper's Table 'Whole'.  Every test below checks the oracle against
something other than itself: hand-worked values, closed forms, invariants,
exhaustive brute force by dense reachability (Eqs. 14-17, the Normalizer of
(A+I)^N with N >= n) and scipy's connected components.
"""
import itertools
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
import synth
from synth.graphs import disjoint_union

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pc_worked_examples.json")


def both(g, genes):
    a = oracle.pc(g.row_ptr, g.col, np.asarray(genes, dtype=np.int32), "bfs")
    b = oracle.pc(g.row_ptr, g.col, np.asarray(genes, dtype=np.int32), "uf")
    return a, b


def test_worked_examples():
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        e = np.array(case["edges"], dtype=np.int64).reshape(-1, 2)
        g = synth.csr_from_edges(case["n"], e[:, 0], e[:, 1])
        for s in case["sets"]:
            a, b = both(g, s["del"])
            assert a == s["pc"], (case["name"], s)
            assert b == s["pc"], (case["name"], s)


@pytest.mark.parametrize("g", [synth.ba_graph(300, 2, 5), synth.named_graph("path", 50),
                               synth.named_graph("cycle", 40), synth.named_graph("complete", 30),
                               synth.named_graph("grid", 64)])
def test_k0_connected_is_n_choose_2(g):
    assert both(g, []) == (comb(g.n, 2), comb(g.n, 2))


def test_complete_graph_closed_form():
    g = synth.named_graph("complete", 25)
    rng = np.random.default_rng(3)
    for k in range(0, 26):
        d = rng.choice(25, size=k, replace=False)
        assert both(g, d) == (comb(25 - k, 2), comb(25 - k, 2))


def test_star_closed_form():
    g = synth.named_graph("star", 40)
    assert both(g, [0]) == (0, 0)
    assert both(g, [5, 7, 9]) == (comb(37, 2), comb(37, 2))


def _segments(alive):
    out, run = [], 0
    for a in alive:
        if a:
            run += 1
        elif run:
            out.append(run)
            run = 0
    if run:
        out.append(run)
    return out


def test_path_and_cycle_segments():
    rng = np.random.default_rng(11)
    for n in (2, 7, 31, 200):
        p = synth.named_graph("path", n)
        c = synth.named_graph("cycle", n) if n >= 3 else None
        for k in range(0, min(n, 12)):
            d = rng.choice(n, size=k, replace=False)
            alive = np.ones(n, dtype=bool)
            alive[d] = False
            want = sum(comb(x, 2) for x in _segments(alive))
            assert both(p, d) == (want, want)
            if c is not None:
                if k == 0:
                    want_c = comb(n, 2)
                else:
                    rot = np.roll(alive, -int(d[0]))  # start the walk at a deleted node
                    want_c = sum(comb(x, 2) for x in _segments(rot))
                assert both(c, d) == (want_c, want_c)


def test_disjoint_union_adds():
    g1 = synth.ba_graph(60, 2, 1)
    g2 = synth.er_graph(50, 80, 2)
    g = disjoint_union(g1, g2)
    d1 = np.array([0, 5, 9])
    d2 = np.array([1, 2, 40])
    a = oracle.pc(g1.row_ptr, g1.col, d1) + oracle.pc(g2.row_ptr, g2.col, d2)
    assert both(g, np.concatenate([d1, d2 + g1.n])) == (a, a)


def test_empty_graph_and_duplicates_in_set():
    g = synth.named_graph("empty", 10)
    assert both(g, [1, 2]) == (0, 0)
    g = synth.named_graph("path", 6)
    # a deletion set with a repeated gene is the set of its distinct genes
    assert both(g, [2, 2]) == both(g, [2])


def test_invalid_gene_rejected():
    g = synth.named_graph("path", 6)
    with pytest.raises(oracle.OracleError):
        oracle.pc(g.row_ptr, g.col, [6])
    with pytest.raises(oracle.OracleError):
        oracle.pc(g.row_ptr, g.col, [-1])


def test_invariants_sizes_bound_monotone():
    g = synth.hk_graph(400, 3, 0.3, 2)
    rng = np.random.default_rng(5)
    for _ in range(20):
        k = int(rng.integers(0, 120))
        d = rng.choice(g.n, size=k, replace=False)
        sizes = oracle.component_sizes(g.row_ptr, g.col, d)
        assert sizes.sum() == g.n - k
        pcv = oracle.pc(g.row_ptr, g.col, d)
        assert pcv == sum(comb(int(x), 2) for x in sizes)
        assert pcv <= comb(g.n - k, 2)
        extra = rng.choice(np.setdiff1d(np.arange(g.n), d))
        assert oracle.pc(g.row_ptr, g.col, np.append(d, extra)) <= pcv


def _dense_pc(adj: np.ndarray, alive: np.ndarray) -> np.ndarray:
    """PC by the reachability matrix of Eqs. 14-17: M = Normalizer((A+I)^N), N >= n.

    adj: (n, n) 0/1; alive: (B, n) bool.  Counts connected ordered pairs of
    live nodes, removes the diagonal and halves: PC = (sum M - live) / 2.
    """
    n = adj.shape[0]
    a = adj[None, :, :].astype(np.int64) * alive[:, :, None] * alive[:, None, :]
    m = a + np.eye(n, dtype=np.int64)[None] * alive[:, :, None]
    steps = 0
    while (1 << steps) < n:
        m = np.minimum(m @ m, 1)  # Normalizer after each squaring
        steps += 1
    return (m.sum(axis=(1, 2)) - alive.sum(axis=1)) // 2


@pytest.mark.parametrize("seed,n,edges", [(1, 12, 16), (2, 13, 12), (3, 14, 20), (4, 10, 30)])
def test_exhaustive_all_subsets_against_dense_reachability(seed, n, edges):
    g = synth.er_graph(n, edges, seed)
    adj = np.zeros((n, n), dtype=np.int64)
    u, v = g.edge_list()
    adj[u, v] = 1
    adj[v, u] = 1
    masks = np.arange(1 << n, dtype=np.int64)
    dead = ((masks[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)
    want = _dense_pc(adj, ~dead)
    pop_rows = [np.flatnonzero(row).astype(np.int32) for row in dead]
    # equal-length rows: group subsets by size
    for k in range(n + 1):
        idx = np.flatnonzero(dead.sum(axis=1) == k)
        pop = np.stack([pop_rows[i] for i in idx]) if k > 0 else np.zeros((idx.size, 0), np.int32)
        got_b = oracle.fitness(g.row_ptr, g.col, pop, "bfs")
        got_u = oracle.fitness(g.row_ptr, g.col, pop, "uf")
        assert np.array_equal(got_b, want[idx]), (k,)
        assert np.array_equal(got_u, want[idx]), (k,)


def test_dense_reachability_identity_medium():
    """Eq. 17 on a few hundred nodes with random deletions (N = 2^t >= n)."""
    g = synth.ba_graph(256, 1, 9)  # a tree: deletions split it into many parts
    adj = np.zeros((g.n, g.n), dtype=np.int64)
    u, v = g.edge_list()
    adj[u, v] = 1
    adj[v, u] = 1
    rng = np.random.default_rng(1)
    pops = np.stack([rng.choice(g.n, size=25, replace=False) for _ in range(6)]).astype(np.int32)
    alive = np.ones((6, g.n), dtype=bool)
    for r in range(6):
        alive[r, pops[r]] = False
    assert np.array_equal(oracle.fitness(g.row_ptr, g.col, pops), _dense_pc(adj, alive))


def test_against_scipy_connected_components():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for g in (synth.ba_graph(2000, 2, 3), synth.hk_graph(1500, 2, 0.5, 4),
              synth.rmat_graph(11, 6000, seed=2, chunk=1 << 14)):
        rng = np.random.default_rng(g.n)
        pops = np.stack([rng.choice(g.n, size=g.n // 10, replace=False) for _ in range(5)]).astype(np.int32)
        got = oracle.fitness(g.row_ptr, g.col, pops, "bfs", nthreads=2)
        for r in range(5):
            alive = np.ones(g.n, dtype=bool)
            alive[pops[r]] = False
            keep = np.flatnonzero(alive)
            m = sp.csr_matrix((np.ones(g.col.size), g.col, g.row_ptr), shape=(g.n, g.n))[keep][:, keep]
            _, lab = csgraph.connected_components(m, directed=False)
            sizes = np.bincount(lab)
            assert got[r] == int((sizes.astype(np.int64) * (sizes - 1) // 2).sum())


def test_fitness_threads_agree():
    g = synth.ba_graph(3000, 3, 7)
    pop = synth.random_deletion_sets(g.n, 150, 16, 3)
    a = oracle.fitness(g.row_ptr, g.col, pop, "bfs", nthreads=1)
    b = oracle.fitness(g.row_ptr, g.col, pop, "uf", nthreads=4)
    assert np.array_equal(a, b)


def _dense_mcn(adj, alive):
    """MCN from the reachability matrix of Eq. 17: the largest row sum of Normalizer((A+I)^N) over
    live nodes (end of Section III-C), 0 with no live node."""
    n = adj.shape[0]
    a = adj[None, :, :].astype(np.int64) * alive[:, :, None] * alive[:, None, :]
    m = a + np.eye(n, dtype=np.int64)[None] * alive[:, :, None]
    steps = 0
    while (1 << steps) < n:
        m = np.minimum(m @ m, 1)
        steps += 1
    return m.sum(axis=2).max(axis=1)


@pytest.mark.parametrize("seed,n,edges", [(1, 12, 16), (3, 14, 20), (5, 11, 8)])
def test_mcn_exhaustive_against_dense_reachability(seed, n, edges):
    g = synth.er_graph(n, edges, seed)
    adj = np.zeros((n, n), dtype=np.int64)
    u, v = g.edge_list()
    adj[u, v] = 1
    adj[v, u] = 1
    masks = np.arange(1 << n, dtype=np.int64)
    dead = ((masks[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)
    want = _dense_mcn(adj, ~dead)
    for k in range(n + 1):
        idx = np.flatnonzero(dead.sum(axis=1) == k)
        pop = np.stack([np.flatnonzero(dead[i]).astype(np.int32) for i in idx]) if k > 0 else \
            np.zeros((idx.size, 0), np.int32)
        assert np.array_equal(oracle.fitness(g.row_ptr, g.col, pop, "mcn"), want[idx]), k


def test_mcn_closed_forms():
    path = synth.named_graph("path", 10)
    assert oracle.mcn(path.row_ptr, path.col, []) == 10
    assert oracle.mcn(path.row_ptr, path.col, [4]) == 5  # {0..3} and {5..9}
    assert oracle.mcn(path.row_ptr, path.col, [2, 6]) == 3
    star = synth.named_graph("star", 9)
    assert oracle.mcn(star.row_ptr, star.col, [0]) == 1
    assert oracle.mcn(star.row_ptr, star.col, [1, 2]) == 7
    kn = synth.named_graph("complete", 8)
    assert oracle.mcn(kn.row_ptr, kn.col, [0, 3, 5]) == 5
    assert oracle.mcn(kn.row_ptr, kn.col, list(range(8))) == 0
    both = disjoint_union(synth.named_graph("path", 4), synth.named_graph("cycle", 7))
    assert oracle.mcn(both.row_ptr, both.col, []) == 7
    assert oracle.mcn(both.row_ptr, both.col, [4]) == 6


def test_mcn_against_scipy_and_pc():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = synth.ba_graph(1500, 2, 8)
    rng = np.random.default_rng(2)
    pops = np.stack([rng.choice(g.n, size=200, replace=False) for _ in range(6)]).astype(np.int32)
    got = oracle.fitness(g.row_ptr, g.col, pops, "mcn")
    pc = oracle.fitness(g.row_ptr, g.col, pops)
    for r in range(6):
        alive = np.ones(g.n, dtype=bool)
        alive[pops[r]] = False
        keep = np.flatnonzero(alive)
        m = sp.csr_matrix((np.ones(g.col.size), g.col, g.row_ptr), shape=(g.n, g.n))[keep][:, keep]
        _, lab = csgraph.connected_components(m, directed=False)
        assert got[r] == np.bincount(lab).max()
        c = int(got[r])
        assert c * (c - 1) // 2 <= pc[r]  # the largest component alone contributes C(MCN, 2)


# ---- edge genes (Section III-C: node and edge perturbations both act on the adjacency matrix) ----

def test_edge_fitness_closed_forms():
    n = 9
    path = synth.named_graph("path", n)  # edge i joins i and i+1
    for i in range(n - 1):
        assert oracle.edge_fitness(path.row_ptr, path.col, [i]) == comb(i + 1, 2) + comb(n - i - 1, 2)
        assert oracle.edge_fitness(path.row_ptr, path.col, [i], "mcn") == max(i + 1, n - i - 1)
    cyc = synth.named_graph("cycle", 10)
    assert oracle.edge_fitness(cyc.row_ptr, cyc.col, [3]) == comb(10, 2)  # one cut keeps a cycle connected
    star = synth.named_graph("star", 7)
    assert oracle.edge_fitness(star.row_ptr, star.col, [0, 1, 2]) == comb(4, 2)  # three leaves cut off
    all_edges = list(range(star.num_edges))
    assert oracle.edge_fitness(star.row_ptr, star.col, all_edges) == 0
    assert oracle.edge_fitness(star.row_ptr, star.col, all_edges, "mcn") == 1


def test_node_deletion_equals_removing_its_edges():
    """The paper's statement that deleting a node is removing its incident edges: the deleted
    nodes are left isolated, which adds nothing to PC."""
    g = synth.ba_graph(300, 2, 5)
    u, v = g.edge_list()
    rng = np.random.default_rng(4)
    for _ in range(10):
        genes = rng.choice(g.n, 25, replace=False)
        hit = np.flatnonzero(np.isin(u, genes) | np.isin(v, genes)).astype(np.int32)
        assert oracle.edge_fitness(g.row_ptr, g.col, hit) == oracle.pc(g.row_ptr, g.col, genes)


@pytest.mark.parametrize("seed,n,edges", [(2, 9, 11), (6, 10, 12)])
def test_edge_fitness_exhaustive_against_dense_reachability(seed, n, edges):
    """All 2^E edge subsets: Eq. 17 on the perturbed adjacency matrix (every node alive)."""
    g = synth.er_graph(n, edges, seed)
    u, v = g.edge_list()
    E = u.size
    masks = np.arange(1 << E, dtype=np.int64)
    gone = ((masks[:, None] >> np.arange(E)[None, :]) & 1).astype(bool)
    adj = np.zeros((masks.size, n, n), dtype=np.int64)
    for e in range(E):
        keep = ~gone[:, e]
        adj[keep, u[e], v[e]] = 1
        adj[keep, v[e], u[e]] = 1
    m = adj + np.eye(n, dtype=np.int64)[None]
    steps = 0
    while (1 << steps) < n:
        m = np.minimum(m @ m, 1)
        steps += 1
    want_pc = (m.sum(axis=(1, 2)) - n) // 2
    want_mcn = m.sum(axis=2).max(axis=1)
    for k in range(E + 1):
        idx = np.flatnonzero(gone.sum(axis=1) == k)
        pop = np.stack([np.flatnonzero(gone[i]).astype(np.int32) for i in idx]) if k > 0 else \
            np.zeros((idx.size, 0), np.int32)
        assert np.array_equal(oracle.fitness(g.row_ptr, g.col, pop, "edges"), want_pc[idx]), k
        assert np.array_equal(oracle.fitness(g.row_ptr, g.col, pop, "edges_mcn"), want_mcn[idx]), k
