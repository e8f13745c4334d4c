"""Seeded graph generators producing simple undirected graphs in symmetric CSR.

Shapes follow the critical-node-detection workloads of the GAPA paper (Table of
datasets, Section IV-A: ForestFire, Erdos-Renyi, Barabasi-Albert and Yeast
graphs of a few hundred to a few thousand nodes, mean degree 2-8), which are
not available here; these generators stand in for them at the sizes of the
benchmark configurations.

Readings (the paper does not specify its generators):

* Barabasi-Albert (n, m): seed graph = star on m+1 nodes (centre 0); every
  later node u draws m distinct targets, each uniform over the list that holds
  every endpoint of every edge so far (so proportional to degree), then links
  to them.  Edges = m + (n-m-1)*m.  Node ids are arrival order.
* Holme-Kim (n, m, p) (Holme & Kim, Phys. Rev. E 65, 026107, 2002): seed = m
  isolated nodes whose endpoint list holds each once; node u makes a
  preferential-attachment (PA) link first, then each further link is, with
  probability p, a triad link to a uniform neighbour of the most recent PA
  target that is not yet linked to u (PA when there is none), otherwise a PA
  link to a target not yet linked to u.  Edges = (n-m)*m.
* R-MAT (scale, edges, a, b, c) (Chakrabarti, Zhan and Faloutsos, SDM 2004):
  each sample picks one of four quadrants per level with probabilities
  a, b, c, 1-a-b-c; self-loops are dropped, (u,v) and (v,u) are one edge, and
  samples are drawn until exactly ``edges`` distinct edges exist (kept in order
  of first appearance); then node ids are permuted by a seeded random
  permutation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMixStream, splitmix64


@dataclass
class Graph:
    """Simple undirected graph as symmetric CSR (each edge stored both ways, rows sorted)."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray  # int32[2E]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_edges(self) -> int:
        return int(self.col.shape[0]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64)).astype(np.int32)

    def edge_list(self) -> tuple[np.ndarray, np.ndarray]:
        """Each undirected edge once as (u, v) with u < v, in CSR order."""
        src = np.repeat(np.arange(self.n, dtype=np.int32), self.degrees())
        keep = self.col > src
        return src[keep], self.col[keep]


def csr_from_edges(n: int, u, v, name: str = "", meta: dict | None = None) -> Graph:
    """Symmetric CSR from an undirected edge list; duplicates merged; self-loops rejected."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.shape != v.shape:
        raise ValueError("edge arrays differ in length")
    if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("edge endpoint out of range")
    if np.any(u == v):
        raise ValueError("self-loop in edge list")
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = np.sort(lo * n + hi)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    lo = key // n
    hi = key % n
    arcs = np.concatenate([lo * n + hi, hi * n + lo])
    arcs.sort()
    src = arcs // n
    dst = arcs % n
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for int32 CSR")
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), name, dict(meta or {}))


def ba_graph(n: int, m: int, seed: int = 1) -> Graph:
    """Barabasi-Albert graph (star seed on m+1 nodes, m distinct degree-proportional targets)."""
    if not (1 <= m < n):
        raise ValueError("need 1 <= m < n")
    rs = SplitMixStream(seed ^ 0xBA00000000000000)
    us: list[int] = []
    vs: list[int] = []
    endpoints: list[int] = []
    for leaf in range(1, m + 1):
        us.append(0)
        vs.append(leaf)
        endpoints += (0, leaf)
    for node in range(m + 1, n):
        chosen: list[int] = []
        while len(chosen) < m:
            t = endpoints[rs.below(len(endpoints))]
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            us.append(node)
            vs.append(t)
            endpoints.append(t)
        endpoints += [node] * m
    return csr_from_edges(n, us, vs, f"ba_n{n}_m{m}_s{seed}", {"kind": "ba", "m": m, "seed": seed})


def hk_graph(n: int, m: int, p: float, seed: int = 1) -> Graph:
    """Holme-Kim power-law cluster graph: PA links mixed with triad links of probability p."""
    if not (1 <= m < n):
        raise ValueError("need 1 <= m < n")
    rs = SplitMixStream(seed ^ 0x4B00000000000000)
    adj: list[list[int]] = [[] for _ in range(n)]
    us: list[int] = []
    vs: list[int] = []
    endpoints: list[int] = list(range(m))

    def pa_target(linked: set) -> int:
        while True:
            t = endpoints[rs.below(len(endpoints))]
            if t not in linked:
                return t

    for node in range(m, n):
        linked: set = set()
        targets: list[int] = []
        last_pa = pa_target(linked)
        linked.add(last_pa)
        targets.append(last_pa)
        while len(targets) < m:
            if rs.unit() < p:
                cands = [w for w in adj[last_pa] if w not in linked]
                if cands:
                    w = cands[rs.below(len(cands))]
                    linked.add(w)
                    targets.append(w)
                    continue
            last_pa = pa_target(linked)
            linked.add(last_pa)
            targets.append(last_pa)
        for t in targets:
            us.append(node)
            vs.append(t)
            adj[node].append(t)
            adj[t].append(node)
            endpoints.append(t)
        endpoints += [node] * m
    return csr_from_edges(n, us, vs, f"hk_n{n}_m{m}_p{p}_s{seed}", {"kind": "hk", "m": m, "p": p, "seed": seed})


def _below_vec(words: np.ndarray, bound: int) -> np.ndarray:
    return ((words >> np.uint64(32)) * np.uint64(bound)) >> np.uint64(32)


def random_permutation(n: int, seed: int) -> np.ndarray:
    """Uniform random permutation of range(n): argsort of n SplitMix64 keys (stable)."""
    keys = splitmix64(seed ^ 0x5045524D00000000, 0, n)
    return np.argsort(keys, kind="stable").astype(np.int64)


def relabel(g: Graph, seed: int) -> Graph:
    """The same graph with node ids permuted by a seeded random permutation."""
    perm = random_permutation(g.n, seed)  # old id -> new id
    u, v = g.edge_list()
    return csr_from_edges(g.n, perm[u], perm[v], g.name + f"_perm{seed}", dict(g.meta, relabel=seed))


def _rmat_keys(scale: int, count: int, ta, tb, tc, stream: int) -> np.ndarray:
    """Samples 0..count-1: edge keys min*n+max, or -1 for self-loops."""
    n = 1 << scale
    u = np.zeros(count, dtype=np.int64)
    v = np.zeros(count, dtype=np.int64)
    for lvl in range(scale):
        # one SplitMix64 stream per recursion level; sample j uses value j of each
        w = splitmix64(stream ^ (lvl << 48), 0, count) >> np.uint64(32)
        u = (u << 1) | (w >= tb).astype(np.int64)  # quadrants c, d set the row bit
        v = (v << 1) | (((w >= ta) & (w < tb)) | (w >= tc)).astype(np.int64)  # quadrants b, d set the column bit
    key = np.minimum(u, v) * n + np.maximum(u, v)
    key[u == v] = -1
    return key


def rmat_graph(scale: int, edges: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 1, permute: bool = True, chunk: int | None = None) -> Graph:
    """R-MAT graph with exactly ``edges`` distinct undirected non-loop edges on 2^scale nodes."""
    n = 1 << scale
    if edges > n * (n - 1) // 2:
        raise ValueError("more edges than a simple graph can hold")
    ta = np.uint64(int(a * 4294967296.0))
    tb = np.uint64(int((a + b) * 4294967296.0))
    tc = np.uint64(int((a + b + c) * 4294967296.0))
    stream = seed ^ 0x524D415400000000
    count = max(1024, int(edges * 1.3))
    while True:
        key = _rmat_keys(scale, count, ta, tb, tc, stream)
        order = np.argsort(key, kind="stable")  # equal keys keep sample order
        sk = key[order]
        first = np.concatenate(([True], sk[1:] != sk[:-1])) & (sk >= 0)
        first_idx = np.sort(order[first])  # first appearance of every distinct edge, in sample order
        if first_idx.size >= edges:
            break
        count = int(count * 1.25) + 1024
    keys = key[first_idx[:edges]]
    lo = keys // n
    hi = keys % n
    if permute:
        perm = random_permutation(n, seed)
        lo, hi = perm[lo], perm[hi]
    return csr_from_edges(n, lo, hi, f"rmat_s{scale}_e{edges}_s{seed}",
                          {"kind": "rmat", "a": a, "b": b, "c": c, "seed": seed, "samples": int(first_idx[edges - 1]) + 1})


def er_graph(n: int, m_edges: int, seed: int = 1) -> Graph:
    """Erdos-Renyi G(n, M): M distinct edges drawn uniformly (first appearance order)."""
    if m_edges > n * (n - 1) // 2:
        raise ValueError("too many edges")
    rs = SplitMixStream(seed ^ 0x4552000000000000)
    seen: set = set()
    us: list[int] = []
    vs: list[int] = []
    while len(us) < m_edges:
        x = rs.below(n)
        y = rs.below(n)
        if x == y:
            continue
        key = (min(x, y), max(x, y))
        if key in seen:
            continue
        seen.add(key)
        us.append(key[0])
        vs.append(key[1])
    return csr_from_edges(n, us, vs, f"er_n{n}_m{m_edges}_s{seed}", {"kind": "er", "seed": seed})


def named_graph(kind: str, n: int, **kw) -> Graph:
    """Small graphs with known structure: path, cycle, star, complete, empty, grid, two_cliques."""
    if kind == "path":
        u = np.arange(n - 1)
        return csr_from_edges(n, u, u + 1, f"path{n}")
    if kind == "cycle":
        u = np.arange(n)
        return csr_from_edges(n, u, (u + 1) % n, f"cycle{n}")
    if kind == "star":
        return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), f"star{n}")
    if kind == "complete":
        iu = np.triu_indices(n, 1)
        return csr_from_edges(n, iu[0], iu[1], f"K{n}")
    if kind == "empty":
        return csr_from_edges(n, [], [], f"empty{n}")
    if kind == "grid":
        w = kw.get("width", int(math.isqrt(n)))
        h = n // w
        us, vs = [], []
        for r in range(h):
            for cidx in range(w):
                x = r * w + cidx
                if cidx + 1 < w:
                    us.append(x)
                    vs.append(x + 1)
                if r + 1 < h:
                    us.append(x)
                    vs.append(x + w)
        return csr_from_edges(w * h, us, vs, f"grid{w}x{h}")
    raise ValueError(f"unknown graph kind {kind}")


def disjoint_union(*graphs: Graph) -> Graph:
    """Disjoint union, node ids offset in argument order."""
    us, vs = [], []
    off = 0
    for g in graphs:
        u, v = g.edge_list()
        us.append(u.astype(np.int64) + off)
        vs.append(v.astype(np.int64) + off)
        off += g.n
    return csr_from_edges(off, np.concatenate(us) if us else [], np.concatenate(vs) if vs else [],
                          "+".join(g.name for g in graphs))


def batched_instances(count: int = 64, seed: int = 0, n_lo: int = 500, n_hi: int = 50000,
                      pops=(32, 64, 128, 256, 512)) -> list[dict]:
    """Instance draws of the batched workload: n log-uniform in [n_lo, n_hi], m in 2..5,
    population from ``pops``, k = round(0.05 n); graph seed = instance index + 1."""
    out = []
    for i in range(count):
        w = splitmix64(seed ^ 0x4241544300000000, 3 * i, 3)
        u = float(w[0] >> np.uint64(11)) * (1.0 / (1 << 53))
        n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        m = 2 + int(_below_vec(w[1:2], 4)[0])
        s = pops[int(_below_vec(w[2:3], len(pops))[0])]
        out.append({"index": i, "n": n, "m": m, "pop": s, "k": int(round(0.05 * n)), "graph_seed": i + 1})
    return out
