"""Plain fp64 reference of the fitness surrogate (test infrastructure only).

The surrogate is not part of the paper: it pre-screens children so that only
the most promising fraction gets the exact pairwise-connectivity fitness of
Section III-C.  Definition shared with the CUDA implementation:

  features of a deletion set D (k genes) on a graph with degrees d and E edges
    e(D)  = (1 / sqrt(k)) * sum_{v in D} Emb[v]                 (64 values)
    q_v   = log1p(d_v);  f1 = mean q, f2 = max q,
    f3    = sqrt(max(mean q^2 - f1^2, 0)),  f4 = sum d_v / (2E)
    residual degrees of the live nodes u (u not in D) adjacent to D, in G[V - D]:
    r0    = #{u : some neighbour in D, no live neighbour}      (isolated by the deletion)
    r1    = #{u : some neighbour in D, exactly one live one}   (made pendant by the deletion)
    r2    = #{components of G[V - D] of exactly two nodes, one of them adjacent to D}
    f5    = log1p(r0),  f6 = log1p(r1),  f7 = log1p(r2)
    z_j   = (r_j - m_j) / max(s_j, 1) for j = 0, 1, 2, where m_j and s_j are the
            mean and the population standard deviation of r_j over the rows
            scored together (one generation's children, or one training
            batch), so that z compares a child with its siblings
    x     = [e(D), f1, f2, f3, f4, f5, f6, f7, z0, z1, z2, 0 x 6]  (80 values)

  On sparse graphs most children of one generation share the giant
  component's size up to a few nodes that the deletion isolates, so their
  pairwise connectivity is ordered by r0 and r2 (an isolated node removes
  about n pairs from the giant component, an isolated pair about 2n); r1
  counts the nodes one more deletion would isolate.  The counts drift upward
  over a run while the differences between siblings stay a few units, so the
  log1p values squeeze those differences late in a run; z keeps them at a
  fixed scale, matching the sibling-relative training target.
  model   z1 = x W1 + b1, h1 = relu(z1)   (W1: 80 x 256)
          z2 = h1 W2 + b2, h2 = relu(z2)  (W2: 256 x 256)
          y  = h2 . w3 + b3
  loss    mean over the batch of (y - t)^2
  AdamW   (Loshchilov & Hutter, ICLR 2019) on every parameter, step tau >= 1:
          m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
          p = p - lr * ( (m / (1 - b1^tau)) / (sqrt(v / (1 - b2^tau)) + eps) + wd * p )

Parameters are a dict of numpy arrays: W1 (80, 256), b1 (256,), W2 (256, 256),
b2 (256,), w3 (256,), b3 (1,), E (n, 64).
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, EMB = 80, 256, 64


def degrees_from_csr(row_ptr) -> np.ndarray:
    return np.diff(np.asarray(row_ptr, dtype=np.int64)).astype(np.float64)


def residual_degree_counts(row_ptr, col, genes) -> tuple[int, int, int]:
    """(r0, r1, r2): live nodes adjacent to the deletion set left with no live neighbour, and with
    exactly one; and two-node components of G[V - D] with a node adjacent to the deletion set."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = row_ptr.size - 1
    dead = np.zeros(n, dtype=bool)
    dead[np.asarray(genes, dtype=np.int64)] = True
    owner = np.repeat(np.arange(n), np.diff(row_ptr))
    dead_arc = dead[np.asarray(col)]
    live_nb = np.bincount(owner, weights=(~dead_arc).astype(np.float64), minlength=n)
    dead_nb = np.bincount(owner, weights=dead_arc.astype(np.float64), minlength=n)
    touched = ~dead & (dead_nb > 0)
    r0 = int(np.count_nonzero(touched & (live_nb == 0)))
    r1 = int(np.count_nonzero(touched & (live_nb == 1)))
    # two-node components: a live arc (u, w), u < w, whose ends have exactly one live neighbour each
    colv = np.asarray(col, dtype=np.int64)
    arc = (owner < colv) & ~dead[owner] & ~dead[colv] & (live_nb[owner] == 1) & (live_nb[colv] == 1)
    arc &= (dead_nb[owner] > 0) | (dead_nb[colv] > 0)
    r2 = int(np.count_nonzero(arc))
    return r0, r1, r2


def features(pop: np.ndarray, E: np.ndarray, row_ptr, col) -> np.ndarray:
    """x for every row of pop (int32[s][k]) on the CSR graph (row_ptr, col) -> float64[s][80]."""
    pop = np.asarray(pop)
    s, k = pop.shape
    deg = degrees_from_csr(row_ptr)
    num_edges = np.asarray(col).size // 2
    x = np.zeros((s, IN), dtype=np.float64)
    q = np.log1p(deg)
    counts = np.zeros((s, 3), dtype=np.int64)
    for i in range(s):
        genes = pop[i]
        x[i, :EMB] = E[genes].sum(axis=0) / np.sqrt(k)
        qi = q[genes]
        f1 = qi.mean()
        x[i, 64] = f1
        x[i, 65] = qi.max()
        x[i, 66] = np.sqrt(max((qi * qi).mean() - f1 * f1, 0.0))
        x[i, 67] = deg[genes].sum() / (2.0 * num_edges)
        r0, r1, r2 = residual_degree_counts(row_ptr, col, genes)
        counts[i] = (r0, r1, r2)
        x[i, 68] = np.log1p(r0)
        x[i, 69] = np.log1p(r1)
        x[i, 70] = np.log1p(r2)
    x[:, 71:74] = standardised_counts(counts)
    return x


def standardised_counts(counts: np.ndarray) -> np.ndarray:
    """z_j = (r_j - mean_j) / max(sd_j, 1) per column of counts (int[s][3]), the mean and the
    population standard deviation taken over the s rows; float32 values, as the model reads them."""
    counts = np.asarray(counts, dtype=np.int64)
    z = np.zeros(counts.shape, dtype=np.float64)
    rows = counts.shape[0]
    if rows == 0:
        return z
    for j in range(counts.shape[1]):
        c = counts[:, j]
        mean = float(c.sum()) / rows
        var = float((c * c).sum()) / rows - mean * mean
        sd = max(np.sqrt(max(var, 0.0)), 1.0)
        z[:, j] = ((c - mean) / sd).astype(np.float32)
    return z


def forward(params: dict, x: np.ndarray) -> tuple[np.ndarray, dict]:
    z1 = x @ params["W1"] + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"] + params["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ params["w3"] + params["b3"][0]
    return y, {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def loss_and_grads(params: dict, pop: np.ndarray, t: np.ndarray, row_ptr, col):
    """MSE loss of the batch and the gradient of every parameter (fp64)."""
    k = pop.shape[1]
    x = features(pop, params["E"], row_ptr, col)
    y, c = forward(params, x)
    B = y.shape[0]
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / B
    g = {"w3": c["h2"].T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, params["w3"]) * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"].T) * (c["z1"] > 0)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    dx = dz1 @ params["W1"].T
    gE = np.zeros_like(params["E"])
    for b in range(B):
        np.add.at(gE, pop[b], dx[b, :EMB] / np.sqrt(k))
    g["E"] = gE
    return loss, g, y


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (8 significant bits, ties to even) via the float32 bit
    pattern: add 0x7FFF plus the lowest kept bit, drop the low 16 bits; returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grads_stored(params: dict, pop: np.ndarray, t, row_ptr, col, rnd=round_bf16):
    """loss_and_grads with `rnd` applied to every tensor the GPU keeps in BF16: the embedding
    table, the features, W1, W2, the activations h1 and h2 and the backward signals dz2 and dz1
    (products and sums in fp64, as the GPU accumulates in FP32).  With rnd = identity it is
    loss_and_grads.  t = None gives the scores only: (None, None, y)."""
    k = pop.shape[1]
    x = rnd(features(pop, rnd(params["E"]), row_ptr, col))
    W1, W2 = rnd(params["W1"]), rnd(params["W2"])
    z1 = x @ W1 + params["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + params["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    y = h2 @ params["w3"] + params["b3"][0]
    if t is None:
        return None, None, y
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / y.shape[0]
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = rnd(np.outer(dy, params["w3"]) * (z2 > 0))
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = rnd((dz2 @ W2.T) * (z1 > 0))
    g["W1"] = x.T @ dz1
    g["b1"] = np.sum(dz1, axis=0)
    dx = dz1 @ W1.T
    gE = np.zeros_like(params["E"])
    for b in range(y.shape[0]):
        np.add.at(gE, pop[b], dx[b, :EMB] / math.sqrt(k))
    g["E"] = gE
    return loss, g, y


def adamw_step(params: dict, grads: dict, state: dict, tau: int, lr=1e-3, b1=0.9, b2=0.999, wd=0.01, eps=1e-8):
    """One AdamW step in place; state holds m and v per parameter."""
    for name, p in params.items():
        gr = grads[name]
        m = state.setdefault(("m", name), np.zeros_like(p))
        v = state.setdefault(("v", name), np.zeros_like(p))
        m *= b1
        m += (1 - b1) * gr
        v *= b2
        v += (1 - b2) * gr * gr
        mh = m / (1 - b1 ** tau)
        vh = v / (1 - b2 ** tau)
        p -= lr * (mh / (np.sqrt(vh) + eps) + wd * p)


def spearman(a, b) -> float:
    """Spearman rank correlation (average ranks for ties)."""
    def ranks(x):
        x = np.asarray(x, dtype=np.float64)
        order = np.argsort(x, kind="stable")
        r = np.empty_like(x)
        r[order] = np.arange(x.size, dtype=np.float64)
        # average ties
        xs = x[order]
        i = 0
        while i < x.size:
            j = i
            while j + 1 < x.size and xs[j + 1] == xs[i]:
                j += 1
            if j > i:
                r[order[i:j + 1]] = (i + j) / 2.0
            i = j + 1
        return r
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0
