"""A sequential model of the forest-piece evaluation of one member (the decomposition used by the
forest-piece fitness kernel), checked against the oracle on the CPU.

The fitness is PC (or MCN) of G[V minus D] (Section III-C, Eq. 13; PC(G) of Table "Whole").  The
forest-piece evaluation keeps no label per node:
* A forest in BFS numbering (every parent precedes its child) gives every node its subtree size
  and a preorder position, so that a subtree is an interval of positions.  With the top hubs
  numbered last, a component may hold several trees.
* Deleting D cuts the forest into pieces rooted at the live children of deleted nodes ("tops")
  and at the live roots of every tree of a component holding deleted nodes; a component without
  deleted nodes stays whole.
* A piece's size is its root's subtree size less the subtrees of the deleted nodes whose parent
  lies in the piece.
* Each top re-picks a live lower-numbered neighbour and unites with that node's piece.
* Only the live nodes of pieces outside the largest class scan their arcs; each arc to a live node
  of another piece unites the two classes.

The central claims are that the subtraction gives every piece's exact node count, and that
scanning only outside the giant class yields the components of G[V minus D].  This file checks
both against a BFS of G[V minus D] and the oracle, on random and hub-heavy deletion sets and on
graphs of several components.  No GPU is touched.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.graphs import disjoint_union


def forest(g, hubs_last=0):
    """BFS numbering from the highest-degree node of each component (with hubs_last, the top hubs
    by degree are left out of the BFS and numbered last, by their lowest-numbered neighbour);
    parents are each node's lowest-numbered neighbour when that one is lower, so they precede
    their children.  With hubs last, a hub whose neighbours all come later starts a tree of its
    own inside a larger component, so components are taken from the edges."""
    n = g.n
    deg = g.degrees()
    hub = set(np.argsort(-deg, kind="stable")[:hubs_last].tolist())
    num = [-1] * n
    order = []
    for s in [int(np.argmax(deg))] + list(range(n)):
        if num[s] >= 0 or s in hub:
            continue
        num[s] = len(order)
        order.append(s)
        head = num[s]
        while head < len(order):
            u = order[head]
            head += 1
            for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                w = int(w)
                if num[w] < 0 and w not in hub:
                    num[w] = len(order)
                    order.append(w)
    late = sorted(hub, key=lambda h: (min([num[int(w)] for w in g.col[g.row_ptr[h]:g.row_ptr[h + 1]]
                                           if num[int(w)] >= 0], default=n), h))
    for h in late:
        num[h] = len(order)
        order.append(h)
    adj = [sorted(num[int(w)] for w in g.col[g.row_ptr[order[x]]:g.row_ptr[order[x] + 1]]) for x in range(n)]
    tp = [min([a for a in adj[x] if a < x], default=x) for x in range(n)]
    kids = [[] for _ in range(n)]
    for x in range(n):
        if tp[x] != x:
            kids[tp[x]].append(x)
    sz = [1] * n
    for x in range(n - 1, -1, -1):
        if tp[x] != x:
            sz[tp[x]] += sz[x]
    pre, at, root, nxt, cursor = [0] * n, [0] * n, [0] * n, [0] * n, 0
    for x in range(n):  # children in ascending order, trees by ascending root
        p = tp[x]
        if p == x:
            pre[x], cursor, root[x] = cursor, cursor + sz[x], x
        else:
            pre[x] = nxt[p]
            nxt[p] += sz[x]
            root[x] = root[p]
        nxt[x] = pre[x] + 1
        at[pre[x]] = x
    # components: the trees joined by edges; representative = smallest root
    uf = list(range(n))

    def find(x):
        while uf[x] != x:
            x = uf[x]
        return x

    for x in range(n):
        for a in adj[x]:
            ra, rb = find(root[x]), find(root[a])
            if ra != rb:
                uf[max(ra, rb)] = min(ra, rb)
    crep = [find(root[x]) for x in range(n)]
    csize = [0] * n
    for x in range(n):
        csize[crep[x]] += 1
    croots = {}
    for x in range(n):
        if tp[x] == x:
            croots.setdefault(crep[x], []).append(x)
    return dict(num=num, tp=tp, adj=adj, kids=kids, sz=sz, pre=pre, at=at, crep=crep, csize=csize, croots=croots)


def c2(x):
    return x * (x - 1) // 2


def piece_eval(F, genes, objective="pc"):
    """The forest-piece evaluation; returns (objective, pieces, sizes of every piece)."""
    tp, adj, kids, sz, pre, at, crep = (F[k] for k in ("tp", "adj", "kids", "sz", "pre", "at", "crep"))
    n = len(tp)
    dead = [False] * n
    dl = []
    for d in genes:
        b = F["num"][int(d)]
        if not dead[b]:
            dead[b] = True
            dl.append(b)
    if len(dl) == n:
        return 0, [], []
    seen = set()
    pn, pw, ps = [], [], []
    for b in dl:
        rep = crep[b]
        if rep not in seen:  # every tree of a touched component gives a piece at its live root
            seen.add(rep)
            for r in F["croots"][rep]:
                if not dead[r]:
                    pn.append(r), pw.append(r), ps.append(sz[r])
        for c in kids[b]:
            if dead[c]:
                continue
            w = next((a for a in adj[c] if a < c and not dead[a]), c)
            pn.append(c), pw.append(w), ps.append(sz[c])
    pid = {c: i for i, c in enumerate(pn)}

    def walk(y):
        while tp[y] != y and not dead[tp[y]]:
            y = tp[y]
        return y

    for b in dl:
        if tp[b] != b and not dead[tp[b]]:
            ps[pid[walk(tp[b])]] -= sz[b]
    uf = list(range(len(pn)))

    def find(x):
        while uf[x] != x:
            uf[x] = uf[uf[x]]
            x = uf[x]
        return x

    def unite(a, b):
        a, b = find(a), find(b)
        if a != b:
            uf[max(a, b)] = min(a, b)

    for i, w in enumerate(pw):
        if w != pn[i]:
            unite(i, pid[walk(w)])
    acc = {}
    for i in range(len(pn)):
        acc[find(i)] = acc.get(find(i), 0) + ps[i]
    giant = max(acc, key=lambda r: (acc[r], -r)) if acc else -1
    outside = [i for i in range(len(pn)) if find(i) != giant]
    for i in outside:
        c = pn[i]
        for q in range(pre[c], pre[c] + sz[c]):
            x = at[q]
            if dead[x]:
                continue
            y = x
            while y != c and not dead[tp[y]]:
                y = tp[y]
            if y != c:
                continue  # below a deleted node: another piece
            for y in adj[x]:
                if not dead[y]:
                    unite(i, pid[walk(y)])
    acc = {}
    for i in range(len(pn)):
        acc[find(i)] = acc.get(find(i), 0) + ps[i]
    clean = [F["csize"][rep] for rep in F["croots"] if rep not in seen]
    if objective == "mcn":
        return max(list(acc.values()) + clean + [0]), pn, ps
    return sum(c2(v) for v in acc.values()) + sum(c2(v) for v in clean), pn, ps


def piece_of(F, genes):
    """Every live node's piece root, by walking up the forest (the reference for the sizes)."""
    tp = F["tp"]
    dead = set(F["num"][int(d)] for d in genes)
    out = {}
    for x in range(len(tp)):
        if x in dead:
            continue
        y = x
        while tp[y] != y and tp[y] not in dead:
            y = tp[y]
        out[x] = y
    return out


GRAPHS = {
    "ba": lambda: synth.ba_graph(3000, 3, 7),
    "hk": lambda: synth.hk_graph(3000, 4, 0.3, 2),
    "rmat": lambda: synth.rmat_graph(11, 8000, seed=3, chunk=1 << 14),
    "union": lambda: disjoint_union(synth.ba_graph(500, 2, 1), synth.named_graph("path", 300),
                                    synth.named_graph("star", 200), synth.ba_graph(800, 4, 2)),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("hubs", [0, 40])
@pytest.mark.parametrize("hubs_last", [0, 30])
def test_piece_evaluation_equals_oracle(name, hubs, hubs_last):
    g = GRAPHS[name]()
    F = forest(g, hubs_last)
    rng = np.random.default_rng(hubs + 11)
    top = np.argsort(-g.degrees(), kind="stable")
    k = max(1, g.n // 20)
    for r in range(12):
        rest = rng.choice(top[hubs:], k - hubs, replace=False)
        genes = np.concatenate([top[:hubs], rest]).astype(np.int32)
        if r % 3 == 0:
            genes = np.concatenate([genes, genes[:5]])  # repeated genes count once
        pc, pn, ps = piece_eval(F, genes)
        assert pc == oracle.pc(g.row_ptr, g.col, genes), (name, r)
        mcn, _, _ = piece_eval(F, genes, "mcn")
        assert mcn == oracle.mcn(g.row_ptr, g.col, genes), (name, r)
        # the subtraction gives every piece its exact node count
        owner = piece_of(F, genes)
        counts = {}
        for x, c in owner.items():
            counts[c] = counts.get(c, 0) + 1
        for c, size in zip(pn, ps):
            assert counts.get(c, 0) == size, (name, r, c)


def test_hubs_last_forest_has_extra_roots():
    """The hubs-last numbering does start trees inside larger components (the case the
    per-component accounting exists for)."""
    g = GRAPHS["ba"]()
    F = forest(g, 30)
    assert any(len(r) > 1 for r in F["croots"].values())


@pytest.mark.parametrize("hubs_last", [0, 10])
def test_degenerate_sets(hubs_last):
    g = disjoint_union(synth.ba_graph(200, 2, 3), synth.named_graph("path", 50))
    F = forest(g, hubs_last)
    n = g.n
    for genes in ([], [0], list(range(n)), list(range(n - 1)), [int(np.argmax(g.degrees()))] * 3):
        genes = np.array(genes, dtype=np.int32)
        assert piece_eval(F, genes)[0] == oracle.pc(g.row_ptr, g.col, genes)
        assert piece_eval(F, genes, "mcn")[0] == oracle.mcn(g.row_ptr, g.col, genes)
