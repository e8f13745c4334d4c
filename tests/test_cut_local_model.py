"""A sequential model of the cut-local evaluation of one member (the decomposition used by the
shared-memory cut-local fitness kernel), checked against the oracle on the CPU.

The fitness is PC of G[V minus D] (Section III-C, Eq. 13; PC(G) of Table "Whole").  The cut-local
evaluation touches only what the deletion disturbs:
* In BFS numbering from the top hub, a node's tree parent is its lowest-numbered neighbour, and
  the children of a node carry consecutive numbers.
* The live children of deleted nodes ("tops") re-pick their first live lower-numbered neighbour,
  else themselves.
* A top whose root is not R (the first live node) seeds the list of nodes outside R's piece, and
  so does every live component root other than R.  The list then grows down the tree, one level
  at a time.
* The pieces are joined, either along the listed nodes' arcs (a listed end with an unlisted live
  end unites with R directly) or along the non-tree edges with every unlisted live node labelled R.

The central claim is that only listed nodes can end up outside R's component.  This file checks
that claim directly against a BFS of G[V minus D], and checks both join modes against the oracle's
PC, on random and hub-heavy deletion sets and on graphs of several components.  No GPU is touched.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.graphs import disjoint_union


def bfs_numbering(g):
    """BFS from the highest-degree node, then from every node not yet reached; returns the number
    of each original id, the tree parent of each number and the sorted adjacency in numbers."""
    n = g.n
    deg = g.degrees()
    num = [-1] * n
    order, tparent = [], []
    for s in [int(np.argmax(deg))] + list(range(n)):
        if num[s] >= 0:
            continue
        num[s] = len(order)
        order.append(s)
        tparent.append(num[s])
        head = num[s]
        while head < len(order):
            u = order[head]
            head += 1
            for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                w = int(w)
                if num[w] < 0:
                    num[w] = len(order)
                    order.append(w)
                    tparent.append(num[u])
    adj = [sorted(num[int(w)] for w in g.col[g.row_ptr[order[x]]:g.row_ptr[order[x] + 1]]) for x in range(n)]
    return num, tparent, adj


def children_runs(tparent):
    kids = [[] for _ in tparent]
    for x, p in enumerate(tparent):
        if p != x:
            kids[p].append(x)
    return kids


class UF:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        a, b = self.find(a), self.find(b)
        if a != b:
            self.p[max(a, b)] = min(a, b)


def cut_local_pc(tparent, adj, kids, dead, join, seed_component_roots=True):
    """PC of one member by the cut-local decomposition; also returns the listed set."""
    n = len(tparent)
    live = [x not in dead for x in range(n)]
    if not any(live):
        return 0, set()
    R = live.index(True)
    lab = list(tparent)
    tops = [c for d in dead for c in kids[d] if live[c]]
    for c in tops:
        lower = [w for w in adj[c] if w < c and live[w]]
        lab[c] = lower[0] if lower else c

    def root(x):
        while lab[x] != x:
            x = lab[x]
        return x

    seeds = {c for c in tops if root(c) != R}
    if seed_component_roots:
        seeds |= {x for x in range(n) if tparent[x] == x and live[x] and x != R}
    listed, frontier = set(seeds), list(seeds)
    while frontier:  # one tree level per round: live children of listed nodes share their piece
        nxt = [c for x in frontier for c in kids[x] if live[c] and c not in listed]
        listed.update(nxt)
        frontier = nxt
    uf = UF(n)
    for x in range(n):  # a listed node takes its piece root, every other live node R
        if live[x]:
            uf.union(x, root(x) if x in listed else R)
    if join == "scan":
        for x in listed:
            for w in adj[x]:
                if live[w]:
                    uf.union(x, w if w in listed else R)
    else:
        for a in range(n):
            for b in adj[a]:
                if a < b and live[a] and live[b] and tparent[b] != a:  # the non-tree edges
                    uf.union(a, b)
    sizes = {}
    for x in range(n):
        if live[x]:
            r = uf.find(x)
            sizes[r] = sizes.get(r, 0) + 1
    return sum(c * (c - 1) // 2 for c in sizes.values()), listed


def outside_first_live(adj, dead):
    """Live nodes not connected to the first live node (plain BFS of G[V minus D])."""
    n = len(adj)
    live = [x not in dead for x in range(n)]
    if not any(live):
        return set()
    R = live.index(True)
    seen, stack = {R}, [R]
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if live[w] and w not in seen:
                seen.add(w)
                stack.append(w)
    return {x for x in range(n) if live[x] and x not in seen}


GRAPHS = {
    "ba": lambda: synth.ba_graph(300, 2, 1),
    "hk": lambda: synth.hk_graph(300, 3, 0.3, 2),
    "er_sparse": lambda: synth.er_graph(300, 280, 3),  # many components
    "union": lambda: disjoint_union(synth.ba_graph(150, 2, 4), synth.named_graph("path", 60),
                                          synth.named_graph("star", 40), synth.named_graph("empty", 10)),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("kind", ["random", "hubs"])
def test_cut_local_decomposition(name, kind):
    g = GRAPHS[name]()
    num, tparent, adj = bfs_numbering(g)
    n = g.n
    # BFS numbering: every tree parent is the lowest-numbered neighbour, children are consecutive
    for x, p in enumerate(tparent):
        if p != x:
            assert p < x and adj[x][0] == p
    kids = children_runs(tparent)
    for ks in kids:
        assert ks == list(range(ks[0], ks[0] + len(ks))) if ks else True
    rng = np.random.default_rng(len(name) * 7 + (kind == "hubs"))
    k = max(1, n // 10)
    top = np.argsort(-g.degrees(), kind="stable")
    rows = []
    for r in range(12):
        if kind == "hubs":
            h = min(k, 2 + 3 * r)
            rest = rng.choice(top[h:], k - h, replace=False)
            rows.append(np.concatenate([top[:h], rest]))
        else:
            rows.append(rng.choice(n, k, replace=False))
    pop = np.stack(rows).astype(np.int32)
    want = oracle.fitness(g.row_ptr, g.col, pop)
    for i, row in enumerate(pop):
        dead = {num[int(d)] for d in row}
        for join in ("scan", "nontree"):
            pc, listed = cut_local_pc(tparent, adj, kids, dead, join)
            assert pc == want[i], (name, kind, i, join)
        assert outside_first_live(adj, dead) <= listed  # only listed nodes can end outside R's piece


def test_decomposition_edge_cases():
    """All nodes deleted, nothing deleted, and the first live node itself cut off from its tree."""
    g = synth.ba_graph(60, 2, 5)
    num, tparent, adj = bfs_numbering(g)
    kids = children_runs(tparent)
    n = g.n
    assert cut_local_pc(tparent, adj, kids, set(range(n)), "scan")[0] == 0
    pc, listed = cut_local_pc(tparent, adj, kids, set(), "nontree")
    assert pc == n * (n - 1) // 2 and listed == set()
    dead = {0} | set(kids[0])  # the top hub and all its children: R is a grandchild or further
    for join in ("scan", "nontree"):
        pop = np.array([[int(np.flatnonzero(np.array(num) == x)[0]) for x in sorted(dead)]], dtype=np.int32)
        assert cut_local_pc(tparent, adj, kids, dead, join)[0] == oracle.fitness(g.row_ptr, g.col, pop)[0]


def test_model_needs_every_seed():
    """Both kinds of seed matter: without the other components' roots the list misses whole
    components, and the PC of a graph of several components comes out wrong."""
    g = GRAPHS["union"]()
    num, tparent, adj = bfs_numbering(g)
    kids = children_runs(tparent)
    pop = synth.random_deletion_sets(g.n, 20, 6, 3)
    want = oracle.fitness(g.row_ptr, g.col, pop)
    got = [cut_local_pc(tparent, adj, kids, {num[int(d)] for d in row}, "scan", seed_component_roots=False)[0]
           for row in pop]
    assert any(a != b for a, b in zip(got, want))
