"""Pins of the dense SixDST reference (Eqs. 14-17): the exact objectives once N reaches the
diameter, closed forms on paths and stars, and hop-limited breadth-first search on small graphs."""
from collections import deque
from math import comb

import numpy as np
import pytest

import oracle
import synth
from oracle import sixdst_ref as sx


def test_large_n_equals_exact_objectives():
    for seed in range(4):
        g = synth.er_graph(60, 70, seed)
        rng = np.random.default_rng(seed)
        pop = np.stack([rng.choice(g.n, 8, replace=False) for _ in range(5)]).astype(np.int32)
        assert np.array_equal(sx.fitness(g.row_ptr, g.col, pop, hops=g.n), oracle.fitness(g.row_ptr, g.col, pop))
        assert np.array_equal(sx.fitness(g.row_ptr, g.col, pop, hops=g.n, objective="mcn"),
                              oracle.fitness(g.row_ptr, g.col, pop, "mcn"))


def test_one_hop_counts_live_edges():
    g = synth.ba_graph(80, 3, 2)
    u, v = g.edge_list()
    rng = np.random.default_rng(1)
    for _ in range(5):
        genes = rng.choice(g.n, 10, replace=False)
        alive = ~np.isin(np.arange(g.n), genes)
        assert sx.sixdst_fitness(g.row_ptr, g.col, genes, hops=1) == int((alive[u] & alive[v]).sum())


def test_path_and_star_closed_forms():
    n = 20
    path = synth.named_graph("path", n)
    for h in (1, 2, 3, 6, 19):
        assert sx.sixdst_fitness(path.row_ptr, path.col, [], hops=h) == sum(n - d for d in range(1, min(h, n - 1) + 1))
        assert sx.sixdst_fitness(path.row_ptr, path.col, [], hops=h, objective="mcn") == min(n, 2 * h + 1)
    star = synth.named_graph("star", 12)
    assert sx.sixdst_fitness(star.row_ptr, star.col, [], hops=1) == 11
    assert sx.sixdst_fitness(star.row_ptr, star.col, [], hops=2) == comb(12, 2)
    assert sx.sixdst_fitness(star.row_ptr, star.col, [0], hops=6) == 0
    assert sx.sixdst_fitness(star.row_ptr, star.col, [0], hops=6, objective="mcn") == 1


def _ball_counts(g, genes, h):
    dead = set(int(x) for x in genes)
    sizes = []
    for s in range(g.n):
        if s in dead:
            continue
        dist = {s: 0}
        q = deque([s])
        while q:
            x = q.popleft()
            if dist[x] == h:
                continue
            for w in g.col[g.row_ptr[x]:g.row_ptr[x + 1]].tolist():
                if w not in dead and w not in dist:
                    dist[w] = dist[x] + 1
                    q.append(w)
        sizes.append(len(dist))
    return sizes


@pytest.mark.parametrize("h", [1, 2, 3, 6])
def test_hop_limited_bfs(h):
    for seed in range(3):
        g = synth.hk_graph(70, 2, 0.3, seed + 1)
        genes = np.random.default_rng(seed).choice(g.n, 9, replace=False)
        sizes = _ball_counts(g, genes, h)
        assert sx.sixdst_fitness(g.row_ptr, g.col, genes, hops=h) == (sum(sizes) - len(sizes)) // 2
        assert sx.sixdst_fitness(g.row_ptr, g.col, genes, hops=h, objective="mcn") == max(sizes)


def test_monotone_in_hops():
    g = synth.ba_graph(120, 2, 7)
    genes = np.random.default_rng(3).choice(g.n, 12, replace=False)
    vals = [sx.sixdst_fitness(g.row_ptr, g.col, genes, hops=h) for h in range(1, 10)]
    assert all(a <= b for a, b in zip(vals, vals[1:])) and vals[-1] <= oracle.pc(g.row_ptr, g.col, genes)
