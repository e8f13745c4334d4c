"""A sequential model of the sparse (chain-resolving) evaluation of one member, checked against
the oracle on the CPU.  The sparse fitness kernel for graphs whose labels do not fit in shared
memory follows the same steps, with its per-node state in global memory that it clears after use.

The fitness is PC (or MCN) of G[V minus D] (Section III-C, Eq. 13; PC(G) and MCN of Table
"Whole").  In the BFS forest of the upload (numbering from the top hub of each component, so a
node's tree parent is its lowest-numbered neighbour and its children carry consecutive numbers),
deleting D cuts each touched component's tree into pieces: the root's piece (when the root is
live) and one piece below every live child of a deleted node (a "top").  The evaluation never
touches the inside of a piece that stays joined:
* every top re-picks its first live lower-numbered neighbour q (else it is a terminal of its
  own), and its hop is the first top or tree root met walking up the tree from q; hops strictly
  decrease, so following them from any top ends at a terminal: a live tree root or a top that
  re-picked nothing.  Each terminal's set S (the pieces whose chains end at it) is connected;
* terminals form classes: a top that re-picked nothing unites its class with the classes of the
  terminals of its first live neighbours outside its piece (neighbour sampling; any union along
  a live edge is exact, and after the top hub is deleted it saves listing most of the graph);
* per touched component the class of one reference terminal becomes R: the root when it is
  live, else the terminal whose chained tops carry the most subtree nodes (any choice is exact);
* the pieces of every other class are listed (grown down the tree from their tops), the listed
  nodes' arcs unite their classes (an arc to an unlisted live node joins the class to R, since
  every unlisted live node of the component lies in R's class);
* sizes: each class left apart from R counts its listed nodes; R's set is the component's size
  less its deleted nodes less those classes.  PC = the graph's PC less C(size, 2) of every
  touched component plus the new terms.

These tests check the model against the oracle's PC and MCN on random, hub-heavy and dense
deletion sets, graphs of several components, empty and complete deletions, and by exhaustion on
small graphs.  No GPU is touched.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from synth.graphs import disjoint_union


def bfs_forest(g):
    """BFS numbering from the highest-degree node of each component (ties: lower id), as the
    upload builds it; returns the number of every original id, the tree parent of every number
    and the sorted adjacency and lower-neighbour lists in numbers."""
    n = g.n
    deg = g.degrees()
    by_deg = sorted(range(n), key=lambda v: (-int(deg[v]), v))
    num = [-1] * n
    order, tparent = [], []
    for s in by_deg:
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
    lower = [[a for a in adj[x] if a < x] for x in range(n)]
    return num, tparent, adj, lower


class Forest:
    """The upload's per-node tables of the sparse kernel."""

    def __init__(self, g):
        self.n = g.n
        self.num, self.tparent, self.adj, self.lower = bfs_forest(g)
        n = self.n
        self.kids = [[] for _ in range(n)]
        for x, p in enumerate(self.tparent):
            if p != x:
                self.kids[p].append(x)
        for p, ks in enumerate(self.kids):  # children carry consecutive numbers
            assert ks == list(range(ks[0], ks[0] + len(ks))) if ks else True
        self.croot = [0] * n
        for x in range(n):
            p = self.tparent[x]
            self.croot[x] = x if p == x else self.croot[p]
        self.csize = [0] * n
        for x in range(n):
            self.csize[self.croot[x]] += 1
        self.sub = [1] * n
        for x in range(n - 1, -1, -1):
            if self.tparent[x] != x:
                self.sub[self.tparent[x]] += self.sub[x]
        roots = [x for x in range(n) if self.tparent[x] == x]
        self.bysize = sorted(roots, key=lambda r: (-self.csize[r], r))
        self.pc0 = sum(self.csize[r] * (self.csize[r] - 1) // 2 for r in roots)


def sparse_eval(f, dead, objective="pc", stats=None, link=4, link_terminals_only=True):
    """Fitness of the member whose deleted nodes (numbers) are `dead`, by the sparse steps;
    `link`: adjacency entries a top that re-picked nothing samples for links (0: none);
    link_terminals_only=False lets every top chained to such a terminal sample (the kernel
    samples from the terminals only)."""
    n = f.n
    dead = set(dead)
    # tops: the live children of deleted nodes
    tops = [t for d in sorted(dead) for t in f.kids[d] if t not in dead]
    hop = {}
    for t in tops:
        q = t
        for w in f.lower[t]:
            if w not in dead:
                q = w
                break
        y = q
        if q != t:
            while True:
                p = f.tparent[y]
                if p == y or p in dead:
                    break
                y = p
        hop[t] = y
    final = {}
    for t in tops:
        x = hop[t]
        while x in hop and hop[x] != x:
            x = hop[x]
        final[t] = x

    # classes of terminals: union-find, R = None once chosen
    parent = {}

    def find(a):
        while a is not None and parent.get(a, a) != a:
            a = parent[a]
        return a

    def unite(a, b):
        a, b = find(a), find(b)
        if a == b:
            return
        if a is None or b is None:  # R absorbs the other class
            parent[b if a is None else a] = None
        else:  # the larger terminal hooks under the smaller
            parent[max(a, b)] = min(a, b)

    def terminal_of(w):
        y = w
        while True:
            p = f.tparent[y]
            if p == y:
                return y
            if p in dead:
                return final[y]
            y = p

    # sampled links: a top that re-picked nothing unites its class with the classes of its first
    # live neighbours outside its own piece (at most two links)
    for t in tops:
        a = final[t]
        if hop.get(a) != a or (link_terminals_only and a != t):
            continue
        links = 0
        for w in f.adj[t][:link]:
            if links == 2:
                break
            if w in dead or f.tparent[w] == t:
                continue
            b = terminal_of(w)
            if b != a:  # a neighbour chained to the same terminal links nothing
                unite(a, b)
                links += 1
    # reference terminal per touched component
    weight = {}
    for t in tops:
        x = final[t]
        if hop.get(x) == x and f.croot[x] in dead:
            weight[x] = weight.get(x, 0) + f.sub[t]
    ref = {}
    touched = sorted({f.croot[d] for d in dead})
    for c in touched:
        if c not in dead:
            ref[c] = c
    best = {}
    for x in weight:
        c = f.croot[x]
        key = (weight[x], -x)
        if c not in best or key > best[c]:
            best[c] = key
    for c, key in best.items():
        ref[c] = -key[1]
    for c in touched:  # the reference's class becomes R
        if c in ref:
            r = find(ref[c])
            if r is not None:
                parent[r] = None
    # listing: tops whose class is not R, grown down the tree
    cls = {}
    frontier = []
    for t in tops:
        if find(final[t]) is not None:
            cls[t] = final[t]
            frontier.append(t)
    listed = list(frontier)
    while frontier:
        nxt = []
        for u in frontier:
            for x in f.kids[u]:
                if x not in dead:
                    cls[x] = cls[u]
                    nxt.append(x)
        listed += nxt
        frontier = nxt
    # join along the listed nodes' arcs
    for v in listed:
        for w in f.adj[v]:
            if w in dead:
                continue
            unite(cls[v], cls.get(w))  # an unlisted live end lies in R's set
    # sizes
    size = {}
    apart = {}
    for v in listed:
        r = find(cls[v])
        if r is not None:
            size[r] = size.get(r, 0) + 1
            apart[f.croot[v]] = apart.get(f.croot[v], 0) + 1
    ndel = {}
    for d in dead:
        ndel[f.croot[d]] = ndel.get(f.croot[d], 0) + 1
    if stats is not None:
        stats["tops"] = len(tops)
        stats["listed"] = len(listed)
        stats["terminals"] = sum(1 for t in tops if hop[t] == t)
        stats["chained_to_terminals"] = sum(1 for t in tops if hop.get(final[t]) == final[t])
    if objective == "pc":
        pc = f.pc0
        for c in touched:
            rs = f.csize[c] - ndel[c] - apart.get(c, 0)
            pc += rs * (rs - 1) // 2 - f.csize[c] * (f.csize[c] - 1) // 2
        for s in size.values():
            pc += s * (s - 1) // 2
        return pc
    mx = max(size.values(), default=0)
    for c in touched:
        mx = max(mx, f.csize[c] - ndel[c] - apart.get(c, 0))
    touched_set = set(touched)
    for r in f.bysize:  # the largest untouched component
        if r not in touched_set:
            mx = max(mx, f.csize[r])
            break
    return mx


def _members(g, f, sets):
    for genes in sets:
        yield genes, [f.num[int(v)] for v in genes]


def _graphs():
    return [
        ("ba", synth.ba_graph(400, 3, seed=5)),
        ("hk", synth.hk_graph(400, 3, 0.3, seed=6)),
        ("rmat", synth.rmat_graph(9, 2500, seed=7)),
        ("er", synth.er_graph(300, 330, seed=8)),
        ("union", disjoint_union(synth.ba_graph(120, 2, seed=9), synth.named_graph("path", 40),
                                 synth.named_graph("star", 30), synth.er_graph(100, 90, seed=10))),
    ]


@pytest.mark.parametrize("name,g", _graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_sparse_model_random_sets_match_oracle(name, g):
    f = Forest(g)
    rng = np.random.default_rng(11)
    for k in (0, 1, 5, g.n // 20, g.n // 5, g.n // 2):
        for _ in range(6):
            genes = rng.choice(g.n, size=k, replace=False).astype(np.int32)
            dead = [f.num[int(v)] for v in genes]
            assert sparse_eval(f, dead) == oracle.pc(g.row_ptr, g.col, genes), (name, k)
            assert sparse_eval(f, dead, "mcn") == oracle.mcn(g.row_ptr, g.col, genes), (name, k)


@pytest.mark.parametrize("name,g", _graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_sparse_model_hub_heavy_sets_match_oracle(name, g):
    """Deleting the top hubs deletes the tree roots, so the reference is chosen by weight."""
    f = Forest(g)
    order = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(12)
    for hubs in (1, 2, 5, 20, g.n // 10):
        for extra in (0, g.n // 50):
            rest = rng.choice(order[hubs:], size=extra, replace=False)
            genes = np.concatenate([order[:hubs], rest]).astype(np.int32)
            dead = [f.num[int(v)] for v in genes]
            assert sparse_eval(f, dead) == oracle.pc(g.row_ptr, g.col, genes), (name, hubs, extra)
            assert sparse_eval(f, dead, "mcn") == oracle.mcn(g.row_ptr, g.col, genes), (name, hubs, extra)


def test_sparse_model_all_and_none_deleted():
    g = synth.ba_graph(60, 2, seed=13)
    f = Forest(g)
    everything = np.arange(g.n, dtype=np.int32)
    assert sparse_eval(f, [f.num[v] for v in everything]) == 0
    assert sparse_eval(f, [f.num[v] for v in everything], "mcn") == 0
    assert sparse_eval(f, []) == g.n * (g.n - 1) // 2
    assert sparse_eval(f, [], "mcn") == g.n


@pytest.mark.parametrize("name", ["path", "star", "cycle", "complete", "grid"])
def test_sparse_model_all_subsets_of_small_graphs(name):
    g = synth.named_graph(name, 10)
    f = Forest(g)
    for r in range(g.n + 1):
        for genes in itertools.combinations(range(g.n), r):
            genes = np.array(genes, dtype=np.int32)
            dead = [f.num[int(v)] for v in genes]
            assert sparse_eval(f, dead) == oracle.pc(g.row_ptr, g.col, genes), (name, genes)


def test_sparse_model_touches_little_on_random_sets():
    """What the kernel's cost rests on: on random sets of 1 % of a heavy-tailed graph, the tops
    are about one per deleted node and almost nothing is listed."""
    g = synth.rmat_graph(12, 40000, seed=14)
    f = Forest(g)
    rng = np.random.default_rng(15)
    genes = rng.choice(g.n, size=g.n // 100, replace=False)
    st = {}
    assert sparse_eval(f, [f.num[int(v)] for v in genes], stats=st) == oracle.pc(g.row_ptr, g.col, genes.astype(np.int32))
    assert st["tops"] < 4 * len(genes)
    assert st["listed"] < g.n // 20


def test_sparse_model_links_keep_hub_deleting_lists_short():
    """Deleting the top hub (the BFS root) leaves its children chained to hundreds of terminals;
    without the sampled links their whole subtrees would be listed."""
    g = synth.rmat_graph(13, 80000, seed=16)
    f = Forest(g)
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(17)
    genes = np.concatenate([top[:3], rng.choice(top[3:], g.n // 100, replace=False)]).astype(np.int32)
    dead = [f.num[int(v)] for v in genes]
    want = oracle.pc(g.row_ptr, g.col, genes)
    linked, plain, every = {}, {}, {}
    assert sparse_eval(f, dead, stats=linked) == want
    assert sparse_eval(f, dead, stats=plain, link=0) == want
    assert sparse_eval(f, dead, stats=every, link_terminals_only=False) == want
    assert linked["terminals"] > 50
    assert plain["listed"] > 10 * linked["listed"]


def _without_edges_of(g, h):
    """G' = G with every edge of node h removed (h stays, isolated)."""
    u, v = g.edge_list()
    keep = (u != h) & (v != h)
    return synth.csr_from_edges(g.n, u[keep], v[keep])


@pytest.mark.parametrize("name,g", _graphs()[:4], ids=lambda x: x if isinstance(x, str) else "")
def test_sparse_model_on_the_graph_without_the_top_hub(name, g):
    """A member that deletes the top hub h0 has the same PC and MCN on G and on G' = G without h0's
    edges, and on G' the hub is an isolated node, so deleting it cuts nothing in G''s BFS forest: the
    sparse kernel evaluates such members on G''s forest.  Checked on that forest against the
    oracle on G, with h0 alone and with more of the top hubs, and the tops it saves."""
    h0 = int(np.argmax(g.degrees()))
    gp = _without_edges_of(g, h0)
    f, fp = Forest(g), Forest(gp)
    assert fp.tparent[fp.num[h0]] == fp.num[h0] and fp.csize[fp.num[h0]] == 1
    top = np.argsort(-g.degrees(), kind="stable")
    rng = np.random.default_rng(18)
    for hubs in (1, 3, 10):
        rest = rng.choice(top[hubs:], g.n // 20, replace=False)
        genes = np.concatenate([top[:hubs], rest]).astype(np.int32)
        st, stp = {}, {}
        want = oracle.pc(g.row_ptr, g.col, genes)
        assert sparse_eval(f, [f.num[int(v)] for v in genes], stats=st) == want
        assert sparse_eval(fp, [fp.num[int(v)] for v in genes], stats=stp) == want
        assert sparse_eval(fp, [fp.num[int(v)] for v in genes], "mcn") == oracle.mcn(g.row_ptr, g.col, genes)
        if hubs == 1:
            assert stp["tops"] < st["tops"]
