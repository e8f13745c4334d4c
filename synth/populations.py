"""Uniformly random deletion sets (rows of distinct node ids), seeded by SplitMix64."""
from __future__ import annotations

import numpy as np

from .rng import splitmix64


def random_deletion_sets(n: int, k: int, s: int, seed: int = 0) -> np.ndarray:
    """int32[s][k]: row i is a uniformly random k-subset of range(n), in random order.

    Row i takes the k smallest of n SplitMix64 keys from stream (seed, i): a
    uniform subset, independent of the genetic operators' own initialisation.
    """
    if not (0 <= k <= n):
        raise ValueError("need 0 <= k <= n")
    out = np.empty((s, k), dtype=np.int32)
    for i in range(s):
        keys = splitmix64((seed * 0x100000001B3 + i) ^ 0x504F500000000000, 0, n)
        if k == n:
            sel = np.argsort(keys, kind="stable")
        else:
            sel = np.argpartition(keys, k)[:k] if k > 0 else np.empty(0, dtype=np.int64)
            sel = sel[np.argsort(keys[sel], kind="stable")]
        out[i] = sel.astype(np.int32)
    return out
