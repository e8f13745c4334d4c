"""ctypes front end of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline arm are the only callers.  The oracle shares no code with the CUDA
library and never imports it.

All functions take numpy arrays (int32 CSR, int32 populations, int64 fitness)
and raise ``OracleError`` on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
# A prebuilt library to load instead of oracle.c (the planted-mistake tests point this at a copy
# of the oracle with one mistake in it, to show that the pins catch it).
_LIB_OVERRIDE = os.environ.get("GAPA_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

TAG_INIT, TAG_SEL, TAG_XOVER, TAG_MUT, TAG_MUTVAL, TAG_REPAIR, TAG_ROULETTE = 1, 2, 3, 4, 5, 6, 7
FLAG_ROWWISE, FLAG_MU_PLUS_LAMBDA, FLAG_ROULETTE, FLAG_MCN, FLAG_EDGES = 1, 2, 4, 8, 16


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (-O2, OpenMP); returns the path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_components_bfs.argtypes = [i32, P, P, P, i32, P]
        lib.oracle_components_bfs.restype = i64
        lib.oracle_pc_bfs.argtypes = [i32, P, P, P, i32]
        lib.oracle_pc_bfs.restype = i64
        lib.oracle_pc_uf.argtypes = [i32, P, P, P, i32]
        lib.oracle_pc_uf.restype = i64
        lib.oracle_mcn_bfs.argtypes = [i32, P, P, P, i32]
        lib.oracle_mcn_bfs.restype = i64
        lib.oracle_edge_fitness.argtypes = [i32, P, P, P, i32, i32]
        lib.oracle_edge_fitness.restype = i64
        lib.oracle_fitness.argtypes = [i32, P, P, P, i32, i32, P, i32, i32]
        lib.oracle_fitness.restype = ctypes.c_int
        lib.oracle_pop_init.argtypes = [i32, i32, i32, u64, P]
        lib.oracle_pop_init.restype = ctypes.c_int
        lib.oracle_generation.argtypes = [i32, P, P, i32, i32, i32, u32, u32, u64, u32, i32, i32,
                                          P, P, P, P, i32]
        lib.oracle_generation.restype = ctypes.c_int
        lib.oracle_run.argtypes = [i32, P, P, i32, i32, i32, i32, u32, u32, u64, u32, i32,
                                   P, P, P, P, P, i32]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_child_explicit.argtypes = [i32, i32, P, P, P, P, P, P, P]
        lib.oracle_child_explicit.restype = ctypes.c_int
        lib.oracle_uniform_below.argtypes = [u32, i32]
        lib.oracle_uniform_below.restype = i32
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed: int, j: int, i: int, g: int, tag: int, rnd: int = 0) -> int:
    """Word 0 of Philox4x32-10 at counter (j, i, g, tag<<24 | rnd), key = seed."""
    out = philox4x32_10([j, i, g, (tag << 24) | rnd], [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    return int(out[0])


def component_sizes(row_ptr, col, genes) -> np.ndarray:
    row_ptr, col, genes = _i32(row_ptr), _i32(col), _i32(genes)
    n = row_ptr.shape[0] - 1
    sizes = np.zeros(n + 1, dtype=np.int32)
    r = _load().oracle_components_bfs(n, _ptr(row_ptr), _ptr(col), _ptr(genes), genes.shape[0], _ptr(sizes))
    if r < 0:
        raise OracleError(f"components failed with status {r}")
    return sizes[:r].copy()


def pc(row_ptr, col, genes, method: str = "bfs") -> int:
    """Pairwise connectivity of the graph with the genes deleted."""
    row_ptr, col, genes = _i32(row_ptr), _i32(col), _i32(genes)
    n = row_ptr.shape[0] - 1
    f = _load().oracle_pc_bfs if method == "bfs" else _load().oracle_pc_uf
    r = f(n, _ptr(row_ptr), _ptr(col), _ptr(genes), genes.shape[0])
    if r < 0:
        raise OracleError(f"pc failed with status {r}")
    return int(r)


def mcn(row_ptr, col, genes) -> int:
    """Maximum connectivity number: nodes of the largest component with the genes deleted."""
    row_ptr, col, genes = _i32(row_ptr), _i32(col), _i32(genes)
    n = row_ptr.shape[0] - 1
    r = _load().oracle_mcn_bfs(n, _ptr(row_ptr), _ptr(col), _ptr(genes), genes.shape[0])
    if r < 0:
        raise OracleError(f"mcn failed with status {r}")
    return int(r)


def edge_fitness(row_ptr, col, edge_genes, objective: str = "pc") -> int:
    """PC or MCN of the graph with the edges ``edge_genes`` removed; edge ids number the edges
    {u, v}, u < v, in CSR order (u, then v ascending)."""
    row_ptr, col, genes = _i32(row_ptr), _i32(col), _i32(edge_genes)
    n = row_ptr.shape[0] - 1
    r = _load().oracle_edge_fitness(n, _ptr(row_ptr), _ptr(col), _ptr(genes), genes.shape[0],
                                    1 if objective == "mcn" else 0)
    if r < 0:
        raise OracleError(f"edge fitness failed with status {r}")
    return int(r)


def fitness(row_ptr, col, pop, method: str = "bfs", nthreads: int = 1) -> np.ndarray:
    """PC ("bfs", "uf") or MCN ("mcn") of every row of ``pop`` (int32[s][k], node genes), or with
    edge genes PC ("edges") or MCN ("edges_mcn") -> int64[s]."""
    row_ptr, col, pop = _i32(row_ptr), _i32(col), _i32(pop)
    n = row_ptr.shape[0] - 1
    s, k = pop.shape
    fit = np.zeros(s, dtype=np.int64)
    rc = _load().oracle_fitness(n, _ptr(row_ptr), _ptr(col), _ptr(pop), s, k, _ptr(fit),
                                {"bfs": 0, "uf": 1, "mcn": 2, "edges": 3, "edges_mcn": 4}[method], nthreads)
    _check(rc, "fitness")
    return fit


def pop_init(n: int, k: int, s: int, seed: int) -> np.ndarray:
    pop = np.zeros((s, k), dtype=np.int32)
    _check(_load().oracle_pop_init(n, k, s, seed, _ptr(pop)), "pop_init")
    return pop


REPAIR_ROUNDS = 32


def child_explicit(n: int, A, B, from_b, mutated, mutval, later) -> np.ndarray:
    """One child of parents A and B from explicit crossover and mutation masks, the round-0
    candidates ``mutval`` of mutated positions and the repair candidates ``later`` (31 rounds x k)
    - the child assembly and repair of a generation with no random numbers (test entry)."""
    A, B = _i32(A), _i32(B)
    k = A.shape[0]
    fb = np.ascontiguousarray(from_b, dtype=np.uint8)
    mu = np.ascontiguousarray(mutated, dtype=np.uint8)
    mv = _i32(mutval)
    lt = _i32(later).reshape(REPAIR_ROUNDS - 1, k)
    if not (B.shape == fb.shape == mu.shape == mv.shape == (k,)):
        raise ValueError("A, B, from_b, mutated and mutval must all have k entries")
    row = np.full(k, -1, dtype=np.int32)
    _check(_load().oracle_child_explicit(n, k, _ptr(A), _ptr(B), _ptr(fb), _ptr(mu), _ptr(mv),
                                         _ptr(np.ascontiguousarray(lt)), _ptr(row)), "child_explicit")
    return row


def uniform_below(x: int, n: int) -> int:
    """The oracle's map of a 32-bit Philox word to [0, n)."""
    return int(_load().oracle_uniform_below(x & 0xFFFFFFFF, n))


def thresholds(pc_rate: float, pm_rate: float) -> tuple[int, int]:
    """floor(p * 2^32), clamped to 2^32 - 1."""
    f = lambda p: min(int(p * 4294967296.0), 0xFFFFFFFF)
    return f(pc_rate), f(pm_rate)


def generation(row_ptr, col, pop_in, fit_in, g: int, *, tourn: int, pc_thr: int, pm_thr: int,
               seed: int, flags: int = 0, lam: int = 0, nthreads: int = 1):
    row_ptr, col, pop_in = _i32(row_ptr), _i32(col), _i32(pop_in)
    fit_in = np.ascontiguousarray(fit_in, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    s, k = pop_in.shape
    pop_out = np.zeros_like(pop_in)
    fit_out = np.zeros(s, dtype=np.int64)
    rc = _load().oracle_generation(n, _ptr(row_ptr), _ptr(col), k, s, tourn, pc_thr, pm_thr, seed,
                                   flags, g, lam, _ptr(pop_in), _ptr(fit_in), _ptr(pop_out), _ptr(fit_out),
                                   nthreads)
    _check(rc, "generation")
    return pop_out, fit_out


def run(row_ptr, col, *, k: int, pop: int, gens: int, tourn: int, pc_thr: int, pm_thr: int,
        seed: int, flags: int = 0, lam: int = 0, nthreads: int = 1) -> dict:
    row_ptr, col = _i32(row_ptr), _i32(col)
    n = row_ptr.shape[0] - 1
    best = np.zeros(k, dtype=np.int32)
    best_fit = ctypes.c_int64(0)
    traj = np.zeros(gens + 1, dtype=np.int64)
    pop_final = np.zeros((pop, k), dtype=np.int32)
    fit_final = np.zeros(pop, dtype=np.int64)
    rc = _load().oracle_run(n, _ptr(row_ptr), _ptr(col), k, pop, gens, tourn, pc_thr, pm_thr, seed,
                            flags, lam, _ptr(best), ctypes.cast(ctypes.pointer(best_fit), ctypes.c_void_p),
                            _ptr(traj), _ptr(pop_final), _ptr(fit_final), nthreads)
    _check(rc, "run")
    return {"best_set": best, "best_fit": int(best_fit.value), "traj": traj,
            "pop": pop_final, "fit": fit_final}
