"""Plain dense reference of the SixDST reachability fitness (test infrastructure only).

Section III-C, Eqs. 14-17: the perturbation P^(A, p) removes the deleted nodes'
edges (their rows and columns of A become zero), and the accessibility matrix
is M = Normalizer((A + I)^N), where Normalizer sets every non-zero entry to 1:
M[v][u] = 1 exactly when u is within N hops of v in G[V \\ D] (or u = v).  Row v
of M, for a live v, counts the live nodes within N hops of v, itself included;
when N is at least the diameter of every component this is the size of v's
component.  From M:

    PC_N(D)  = (sum over live v of rowsum(v) - live) / 2
    MCN_N(D) = max over live v of rowsum(v)           (0 when no node is live)

so that PC_N = PC and MCN_N = MCN once N reaches every component's diameter.
N = 6 gives the paper's six-degrees-of-separation fitness.  This reference
multiplies N - 1 times and normalises after every product (which leaves the
boolean result of the whole power unchanged); the products run in float64,
exact for 0/1 matrices (sums of at most n < 2^53 ones).
"""
from __future__ import annotations

import numpy as np


def perturbed_adjacency(row_ptr, col, genes) -> tuple[np.ndarray, np.ndarray]:
    """(A with the deleted nodes' rows and columns zeroed, live mask)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.size - 1
    live = np.ones(n, dtype=bool)
    live[np.asarray(genes, dtype=np.int64)] = False
    a = np.zeros((n, n), dtype=np.int64)
    src = np.repeat(np.arange(n), np.diff(row_ptr))
    keep = live[src] & live[col]
    a[src[keep], col[keep]] = 1
    return a, live


def reachability(a: np.ndarray, hops: int) -> np.ndarray:
    """Normalizer((A + I)^hops) by hops - 1 products, normalised after each one."""
    n = a.shape[0]
    base = np.minimum(a + np.eye(n, dtype=np.int64), 1).astype(np.float64)
    m = base.copy()
    for _ in range(hops - 1):
        m = np.minimum(m @ base, 1.0)
    return m.astype(np.int64)


def sixdst_fitness(row_ptr, col, genes, hops: int = 6, objective: str = "pc") -> int:
    a, live = perturbed_adjacency(row_ptr, col, genes)
    m = reachability(a, hops)
    rows = m.sum(axis=1)[live]
    if objective == "mcn":
        return int(rows.max()) if rows.size else 0
    return int((rows.sum() - live.sum()) // 2)


def fitness(row_ptr, col, pop, hops: int = 6, objective: str = "pc") -> np.ndarray:
    return np.array([sixdst_fitness(row_ptr, col, r, hops, objective) for r in np.asarray(pop)], dtype=np.int64)
