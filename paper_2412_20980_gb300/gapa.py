"""Thin ctypes binding of libgapa.so (argument marshalling only).

Every step of the path runs in the library's CUDA kernels; this module checks
dtypes/devices, passes raw pointers and the current torch stream, and turns
status codes into exceptions.  There is no fallback: if libgapa.so is missing
or cannot be loaded, importing the library functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgapa.so")

GAPA_OK = 0
ERRORS = {
    -1: "INVALID_ARG",
    -2: "INVALID_GRAPH",
    -3: "OOM",
    -4: "CUDA",
    -5: "TIMEOUT",
    -6: "STATE",
    -7: "DEVICE",
}
WHERE_HOST, WHERE_DEVICE = 0, 1
FLAG_ROWWISE, FLAG_MU_PLUS_LAMBDA, FLAG_ROULETTE = 1, 2, 4

# every entry point declared in include/gapa.h
EXPORTS = [
    "gapa_create", "gapa_destroy", "gapa_set_stream", "gapa_graph_upload", "gapa_pop_init",
    "gapa_fitness", "gapa_fitness_host", "gapa_generation", "gapa_generation_host", "gapa_run",
    "gapa_sync", "gapa_last_error", "gapa_version", "gapa_profile_begin", "gapa_profile_end",
    "gapa_set_fitness_kernel", "gapa_fitness_noalloc",
    "gapa_batch_create", "gapa_batch_destroy", "gapa_batch_set_teams", "gapa_batch_get_teams",
    "gapa_batch_autotune", "gapa_batch_run",
    "gapa_surrogate_create", "gapa_surrogate_destroy", "gapa_surrogate_predict", "gapa_surrogate_train_step",
    "gapa_surrogate_tensor", "gapa_run_surrogate", "gapa_surrogate_residual", "gapa_offspring",
    "gapa_set_objective", "gapa_set_genes", "gapa_set_sixdst_hops", "gapa_set_sixdst_kernel", "gapa_selftest_wait",
    "gapa_read_bandwidth",
]
FITNESS_AUTO, FITNESS_EDGES, FITNESS_SAMPLED, FITNESS_TREE, FITNESS_TREE_JOIN, FITNESS_TREE_SCAN = 0, 1, 2, 3, 4, 5
FITNESS_TREE_LOCAL = 6
FITNESS_PIECE = 7
FITNESS_SPARSE = 8
OBJECTIVE_PC, OBJECTIVE_MCN, OBJECTIVE_SIXDST_PC, OBJECTIVE_SIXDST_MCN = 0, 1, 2, 3
GENES_NODES, GENES_EDGES = 0, 1


class GapaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Profile(ctypes.Structure):
    """Mirror of gapa_profile."""

    _fields_ = [
        ("fitness_ms", ctypes.c_double),
        ("operators_ms", ctypes.c_double),
        ("fitness_launches", ctypes.c_int64),
        ("operator_launches", ctypes.c_int64),
        ("evals", ctypes.c_int64),
        ("surrogate_ms", ctypes.c_double),
        ("surrogate_launches", ctypes.c_int64),
        ("fitness_calls", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class SurrogateConfig(ctypes.Structure):
    """Mirror of gapa_surrogate_config."""

    _fields_ = [
        ("screened", ctypes.c_int32),
        ("warmup", ctypes.c_int32),
        ("train_steps", ctypes.c_int32),
        ("batch", ctypes.c_int32),
        ("ring", ctypes.c_int32),
        ("lr", ctypes.c_float),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("weight_decay", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("init_scale_emb", ctypes.c_float),
        ("diag_every", ctypes.c_int32),
        ("target_mode", ctypes.c_int32),
    ]


def make_surrogate_config(screened=512, warmup=3, train_steps=4, batch=512, ring=16384, lr=1e-3, beta1=0.9,
                          beta2=0.999, weight_decay=0.01, eps=1e-8, init_scale_emb=0.1, diag_every=0, target_mode=0):
    return SurrogateConfig(screened, warmup, train_steps, batch, ring, lr, beta1, beta2, weight_decay, eps,
                           init_scale_emb, diag_every, target_mode)


class Config(ctypes.Structure):
    """Mirror of gapa_config."""

    _fields_ = [
        ("k", ctypes.c_int32),
        ("pop", ctypes.c_int32),
        ("gens", ctypes.c_int32),
        ("tourn", ctypes.c_int32),
        ("elite", ctypes.c_int32),
        ("pc_thr", ctypes.c_uint32),
        ("pm_thr", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
        ("lam", ctypes.c_int32),
    ]


def threshold(p: float) -> int:
    """floor(p * 2^32), clamped to 2^32 - 1 (a mask bit is set when the draw is below it)."""
    return min(int(p * 4294967296.0), 0xFFFFFFFF)


def make_config(k: int, pop: int, gens: int = 0, tourn: int = 2, pc: float = 0.8, pm: float = 0.02,
                seed: int = 0, flags: int = 0, elite: int = 1, lam: int = 0) -> Config:
    return Config(k, pop, gens, tourn, elite, threshold(pc), threshold(pm), seed & (2**64 - 1), flags, lam)


# GA parameters of the CND algorithms in the paper's parameter table (Table "Params"):
# crossover and mutation rates, iterations, population size and perturbation rate k / n.
PRESETS = {
    "cutoff": {"pc": 0.6, "pm": 0.2, "gens": 5000, "pop": 80, "rate": 0.1},
    "sixdst": {"pc": 0.5, "pm": 0.3, "gens": 5000, "pop": 80, "rate": 0.1},
    "tde": {"pc": 0.5, "pm": 0.3, "gens": 5000, "pop": 10, "rate": 0.1},
}


def preset_config(name: str, n: int, seed: int = 0, tourn: int = 2, flags: int = 0, **overrides) -> Config:
    """A Config with the named preset's rates, iterations and population for a graph of n nodes;
    the budget is k = round(rate * n) (at least 1, below n).  Keyword arguments override fields."""
    p = dict(PRESETS[name])
    p.update(overrides)
    k = min(max(1, int(round(p["rate"] * n))), max(n - 1, 0))
    return make_config(k=p.get("k", k), pop=p["pop"], gens=p["gens"], tourn=tourn, pc=p["pc"], pm=p["pm"],
                       seed=seed, flags=flags)


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libgapa.so (raises OSError when it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"libgapa.so not found at {p}; run paper_2412_20980_gb300.build.build()")
        lib = ctypes.CDLL(p)
        V, I32, I64, U = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
        cfgp = ctypes.POINTER(Config)
        sig = {
            "gapa_create": ([ctypes.POINTER(V), U, V], U),
            "gapa_destroy": ([V], None),
            "gapa_set_stream": ([V, V], U),
            "gapa_graph_upload": ([V, I32, I64, V, V, U], U),
            "gapa_pop_init": ([V, cfgp, V], U),
            "gapa_fitness": ([V, V, I32, I32, V], U),
            "gapa_fitness_host": ([V, V, I32, I32, V], U),
            "gapa_generation": ([V, cfgp, I32, V, V, V, V], U),
            "gapa_generation_host": ([V, cfgp, I32, V, V, V, V], U),
            "gapa_offspring": ([V, cfgp, I32, V, V, V, V], U),
            "gapa_run": ([V, cfgp, V, V, V, V], U),
            "gapa_sync": ([V], U),
            "gapa_profile_begin": ([V], U),
            "gapa_set_fitness_kernel": ([V, U], U),
            "gapa_set_objective": ([V, U], U),
            "gapa_set_genes": ([V, U], U),
            "gapa_set_sixdst_hops": ([V, U], U),
            "gapa_set_sixdst_kernel": ([V, U], U),
            "gapa_selftest_wait": ([V, I64], U),
            "gapa_read_bandwidth": ([V, I64, I32, ctypes.POINTER(ctypes.c_double)], U),
            "gapa_fitness_noalloc": ([U, V, I32, I32, V, V, I32, I32, V], U),
            "gapa_batch_create": ([ctypes.POINTER(V), I32, V, V], U),
            "gapa_batch_destroy": ([V], None),
            "gapa_batch_set_teams": ([V, V], U),
            "gapa_batch_get_teams": ([V, V], U),
            "gapa_batch_autotune": ([V, ctypes.c_char_p], U),
            "gapa_batch_run": ([V, I32, V, V, V], U),
            "gapa_surrogate_create": ([ctypes.POINTER(V), V, ctypes.POINTER(SurrogateConfig), ctypes.c_uint64], U),
            "gapa_surrogate_destroy": ([V], None),
            "gapa_surrogate_predict": ([V, V, I32, I32, V], U),
            "gapa_surrogate_train_step": ([V, V, I32, I32, V, V], U),
            "gapa_surrogate_residual": ([V, V, I32, I32, V], U),
            "gapa_surrogate_tensor": ([V, I32, I32, V, I64, I32], U),
            "gapa_run_surrogate": ([V, cfgp, V, V, V, V, V, V, V, V, I32], U),
            "gapa_profile_end": ([V, ctypes.POINTER(Profile)], U),
            "gapa_last_error": ([], ctypes.c_char_p),
            "gapa_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load().gapa_last_error().decode()


def _check(rc: int):
    if rc != GAPA_OK:
        raise GapaError(rc, last_error())


def _torch():
    import torch

    return torch


def _dev_ptr(t, dtype, name: str, device_index: int):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda or t.device.index != device_index:
        raise ValueError(f"{name} must live on cuda:{device_index}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fitness_noalloc(edges, pop, n: int, out, stream=None):
    """gapa_fitness_noalloc: fitness of pop[s][k] over the device edge list edges[E][2]
    without any allocation by the library; `out` (int64[s] on the same device) is
    caller-provided.  Synchronous."""
    torch = _torch()
    dev = pop.device.index
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    if stream.device.index != dev:
        raise ValueError(f"stream is on cuda:{stream.device.index}, pop on cuda:{dev}")
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must be [E, 2]")
    if pop.dim() != 2:
        raise ValueError("pop must be [s, k]")
    s, k = pop.shape
    if out.dim() != 1 or out.shape[0] < s:
        raise ValueError(f"out must be a 1-D tensor of at least s = {s} elements")
    _check(load().gapa_fitness_noalloc(dev, ctypes.c_void_p(stream.cuda_stream), n, edges.shape[0],
                                       _dev_ptr(edges, torch.int32, "edges", dev),
                                       _dev_ptr(pop, torch.int32, "pop", dev), s, k,
                                       _dev_ptr(out, torch.int64, "fit", dev)))
    return out


class Context:
    """One GPU context holding one uploaded graph (wraps gapa_ctx)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = ctypes.c_void_p()
        _check(self.lib.gapa_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)))
        self.handle = h
        self.n = 0
        self.num_edges = 0
        self._dependents = weakref.WeakSet()  # surrogates built on this context: closed first

    def close(self):
        for dep in list(getattr(self, "_dependents", ())):
            dep.close()
        if getattr(self, "handle", None):
            self.lib.gapa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def stream(self):
        """The torch stream the context borrows (all its work is ordered on it)."""
        return self._stream

    def set_stream(self, stream):
        self._stream = stream
        _check(self.lib.gapa_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    # -- graph -------------------------------------------------------------
    def graph_upload(self, row_ptr, col):
        """Upload a symmetric CSR from numpy (host) or torch (host or this device) int32 arrays."""
        torch = _torch()
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            rp = _dev_ptr(row_ptr, torch.int32, "row_ptr", self.device)
            cp = _dev_ptr(col, torch.int32, "col", self.device)
            n, nnz, where = row_ptr.numel() - 1, col.numel(), WHERE_DEVICE
            keep = (row_ptr, col)
        else:
            rpa = np.ascontiguousarray(row_ptr.numpy() if isinstance(row_ptr, torch.Tensor) else row_ptr, dtype=np.int32)
            ca = np.ascontiguousarray(col.numpy() if isinstance(col, torch.Tensor) else col, dtype=np.int32)
            rp, cp = _host_ptr(rpa), _host_ptr(ca)
            n, nnz, where = rpa.shape[0] - 1, ca.shape[0], WHERE_HOST
            keep = (rpa, ca)
        _check(self.lib.gapa_graph_upload(self.handle, n, nnz, rp, cp, where))
        del keep
        self.n = n
        self.num_edges = nnz // 2

    # -- operators -----------------------------------------------------------
    def pop_init(self, cfg: Config, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((cfg.pop, cfg.k), dtype=torch.int32, device=f"cuda:{self.device}")
        _check(self.lib.gapa_pop_init(self.handle, ctypes.byref(cfg), _dev_ptr(out, torch.int32, "pop", self.device)))
        return out

    def fitness(self, pop, out=None):
        torch = _torch()
        if pop.dim() != 2:
            raise ValueError("pop must be 2-D [s, k]")
        s, k = pop.shape
        if out is None:
            out = torch.empty(s, dtype=torch.int64, device=f"cuda:{self.device}")
        _check(self.lib.gapa_fitness(self.handle, _dev_ptr(pop, torch.int32, "pop", self.device), s, k,
                                     _dev_ptr(out, torch.int64, "fit", self.device)))
        return out

    def fitness_host(self, pop: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        pop = np.ascontiguousarray(pop, dtype=np.int32)
        s, k = pop.shape
        if out is None:
            out = np.empty(s, dtype=np.int64)
        _check(self.lib.gapa_fitness_host(self.handle, _host_ptr(pop), s, k, _host_ptr(out)))
        return out

    def generation(self, cfg: Config, g: int, pop_in, fit_in, pop_out=None, fit_out=None):
        torch = _torch()
        if pop_out is None:
            pop_out = torch.empty_like(pop_in)
        if fit_out is None:
            fit_out = torch.empty_like(fit_in)
        _check(self.lib.gapa_generation(self.handle, ctypes.byref(cfg), g,
                                        _dev_ptr(pop_in, torch.int32, "pop_in", self.device),
                                        _dev_ptr(fit_in, torch.int64, "fit_in", self.device),
                                        _dev_ptr(pop_out, torch.int32, "pop_out", self.device),
                                        _dev_ptr(fit_out, torch.int64, "fit_out", self.device)))
        return pop_out, fit_out

    def offspring(self, cfg: Config, g: int, pop_in, fit_in, pop_out, fit_out):
        """gapa_offspring: the operators of generation g; fit_out[1:] is left for fitness()."""
        torch = _torch()
        _check(self.lib.gapa_offspring(self.handle, ctypes.byref(cfg), g,
                                       _dev_ptr(pop_in, torch.int32, "pop_in", self.device),
                                       _dev_ptr(fit_in, torch.int64, "fit_in", self.device),
                                       _dev_ptr(pop_out, torch.int32, "pop_out", self.device),
                                       _dev_ptr(fit_out, torch.int64, "fit_out", self.device)))
        return pop_out, fit_out

    def generation_host(self, cfg: Config, g: int, pop_in: np.ndarray, fit_in: np.ndarray,
                        pop_out: np.ndarray | None = None, fit_out: np.ndarray | None = None):
        pop_in = np.ascontiguousarray(pop_in, dtype=np.int32)
        fit_in = np.ascontiguousarray(fit_in, dtype=np.int64)
        if pop_out is None:
            pop_out = np.empty_like(pop_in)
        if fit_out is None:
            fit_out = np.empty_like(fit_in)
        _check(self.lib.gapa_generation_host(self.handle, ctypes.byref(cfg), g, _host_ptr(pop_in), _host_ptr(fit_in),
                                             _host_ptr(pop_out), _host_ptr(fit_out)))
        return pop_out, fit_out

    def run(self, cfg: Config, want_pop: bool = False) -> dict:
        torch = _torch()
        best = np.zeros(max(cfg.k, 1), dtype=np.int32)
        best_fit = np.zeros(1, dtype=np.int64)
        traj = np.zeros(cfg.gens + 1, dtype=np.int64)
        pop = torch.empty((cfg.pop, cfg.k), dtype=torch.int32, device=f"cuda:{self.device}") if want_pop else None
        _check(self.lib.gapa_run(self.handle, ctypes.byref(cfg), _host_ptr(best), _host_ptr(best_fit),
                                 _host_ptr(traj),
                                 _dev_ptr(pop, torch.int32, "pop", self.device) if want_pop else None))
        return {"best_set": best[: cfg.k].copy(), "best_fit": int(best_fit[0]), "traj": traj, "pop": pop}

    def sync(self):
        _check(self.lib.gapa_sync(self.handle))

    def set_fitness_kernel(self, variant: int):
        _check(self.lib.gapa_set_fitness_kernel(self.handle, variant))

    def set_genes(self, gene_type: int):
        """GENES_NODES (node ids, the default) or GENES_EDGES (edge ids in CSR order of {u, v}, u < v)."""
        _check(self.lib.gapa_set_genes(self.handle, gene_type))

    def set_objective(self, objective: int):
        """OBJECTIVE_PC (pairwise connectivity, the default), OBJECTIVE_MCN (largest component), or their
        N-hop SixDST forms OBJECTIVE_SIXDST_PC / OBJECTIVE_SIXDST_MCN (dense reachability, Eqs. 14-17)."""
        _check(self.lib.gapa_set_objective(self.handle, objective))

    def selftest_wait(self, spin_limit: int = 1 << 16) -> int:
        """Runs a bounded device-side wait that must time out; returns the library's status code
        (GAPA_ERR_TIMEOUT = -5 expected) without raising."""
        return int(self.lib.gapa_selftest_wait(self.handle, spin_limit))

    def read_bandwidth(self, nbytes: int, reps: int = 10) -> float:
        """gapa_read_bandwidth: GB/s of the fastest of `reps` read passes over an nbytes buffer."""
        out = ctypes.c_double()
        _check(self.lib.gapa_read_bandwidth(self.handle, nbytes, reps, ctypes.byref(out)))
        return float(out.value)

    def set_sixdst_kernel(self, kernel: int):
        """SixDST products (same results): 3 tcgen05 with TMA loads and split roles (the default where
        available), 1 tcgen05 with cp.async loads, 2 tcgen05 with 128-wide tiles only, 0 mma.sync."""
        _check(self.lib.gapa_set_sixdst_kernel(self.handle, kernel))

    def set_sixdst_hops(self, hops: int):
        """N of Normalizer((A + I)^N) for the SixDST objectives (default 6)."""
        _check(self.lib.gapa_set_sixdst_hops(self.handle, hops))

    def profile_begin(self):
        _check(self.lib.gapa_profile_begin(self.handle))

    def profile_end(self) -> dict:
        prof = Profile()
        _check(self.lib.gapa_profile_end(self.handle, ctypes.byref(prof)))
        return prof.as_dict()


class Batch:
    """Many independent GA instances advanced together (wraps gapa_batch).

    `contexts` hold the uploaded graphs (they must outlive the batch); `configs`
    one Config per instance.
    """

    def __init__(self, contexts, configs):
        self.lib = load()
        self.contexts = list(contexts)
        self.configs = list(configs)
        n = len(self.contexts)
        arr = (ctypes.c_void_p * n)(*[c.handle.value for c in self.contexts])
        cfg_arr = (Config * n)(*self.configs)
        self._keep = (arr, cfg_arr)
        h = ctypes.c_void_p()
        _check(self.lib.gapa_batch_create(ctypes.byref(h), n, ctypes.cast(arr, ctypes.c_void_p),
                                          ctypes.cast(cfg_arr, ctypes.c_void_p)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gapa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def teams(self) -> list[int]:
        out = np.zeros(len(self.contexts), dtype=np.int32)
        _check(self.lib.gapa_batch_get_teams(self.handle, _host_ptr(out)))
        return out.tolist()

    @teams.setter
    def teams(self, values):
        arr = np.ascontiguousarray(values, dtype=np.int32)
        _check(self.lib.gapa_batch_set_teams(self.handle, _host_ptr(arr)))

    def autotune(self, cache_path: str | None = None):
        _check(self.lib.gapa_batch_autotune(self.handle, cache_path.encode() if cache_path else None))

    def run(self, gens: int) -> dict:
        num = len(self.contexts)
        best_fit = np.zeros(num, dtype=np.int64)
        ks = [c.k for c in self.configs]
        best_sets = np.zeros(max(1, sum(ks)), dtype=np.int32)
        traj = np.zeros((num, gens + 1), dtype=np.int64)
        _check(self.lib.gapa_batch_run(self.handle, gens, _host_ptr(best_fit), _host_ptr(best_sets), _host_ptr(traj)))
        sets, off = [], 0
        for k in ks:
            sets.append(best_sets[off:off + k].copy())
            off += k
        return {"best_fit": best_fit, "best_sets": sets, "traj": traj}


SURROGATE_TENSORS = {"W1": (0, (80, 256)), "b1": (1, (256,)), "W2": (2, (256, 256)), "b2": (3, (256,)),
                     "w3": (4, (256,)), "b3": (5, (1,)), "E": (6, None)}


class Surrogate:
    """The learned fitness surrogate of a context's graph (wraps gapa_surrogate)."""

    def __init__(self, ctx: "Context", scfg: SurrogateConfig, seed: int = 0):
        self.lib = load()
        self.ctx = ctx
        self.scfg = scfg
        h = ctypes.c_void_p()
        _check(self.lib.gapa_surrogate_create(ctypes.byref(h), ctx.handle, ctypes.byref(scfg), seed & (2**64 - 1)))
        self.handle = h
        ctx._dependents.add(self)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gapa_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, pop, out=None):
        torch = _torch()
        s, k = pop.shape
        if out is None:
            out = torch.empty(s, dtype=torch.float32, device=pop.device)
        _check(self.lib.gapa_surrogate_predict(self.handle, _dev_ptr(pop, torch.int32, "pop", self.ctx.device), s, k,
                                               _dev_ptr(out, torch.float32, "scores", self.ctx.device)))
        return out

    def residual(self, pop, out=None):
        """(r0, r1, r2) residual counts of every row: int32 [rows][3] on the device."""
        torch = _torch()
        s, k = pop.shape
        if out is None:
            out = torch.empty((s, 3), dtype=torch.int32, device=pop.device)
        _check(self.lib.gapa_surrogate_residual(self.handle, _dev_ptr(pop, torch.int32, "pop", self.ctx.device), s,
                                                k, _dev_ptr(out, torch.int32, "counts", self.ctx.device)))
        return out

    def train_step(self, pop, target) -> float:
        torch = _torch()
        s, k = pop.shape
        loss = ctypes.c_float(0.0)
        _check(self.lib.gapa_surrogate_train_step(self.handle, _dev_ptr(pop, torch.int32, "pop", self.ctx.device), s,
                                                  k, _dev_ptr(target, torch.float32, "target", self.ctx.device),
                                                  ctypes.byref(loss)))
        return float(loss.value)

    def _shape(self, name):
        which, shape = SURROGATE_TENSORS[name]
        return which, (shape if shape is not None else (self.ctx.n, 64))

    def tensor(self, name: str, grad: bool = False) -> np.ndarray:
        which, shape = self._shape(name)
        out = np.zeros(shape, dtype=np.float32)
        _check(self.lib.gapa_surrogate_tensor(self.handle, which, int(grad), _host_ptr(out), out.size, 0))
        return out

    def set_tensor(self, name: str, value: np.ndarray):
        which, shape = self._shape(name)
        arr = np.ascontiguousarray(value, dtype=np.float32).reshape(shape)
        _check(self.lib.gapa_surrogate_tensor(self.handle, which, 0, _host_ptr(arr), arr.size, 1))

    def params(self) -> dict:
        return {name: self.tensor(name).astype(np.float64) for name in SURROGATE_TENSORS}


def run_surrogate(ctx: "Context", cfg: Config, sg: "Surrogate | None" = None, diag_cap: int = 0) -> dict:
    """gapa_run_surrogate: the surrogate-screened (mu+lambda) run, or the plain one with sg=None."""
    G = cfg.gens
    best_fit = np.zeros(1, dtype=np.int64)
    best = np.zeros(max(1, cfg.k), dtype=np.int32)
    traj = np.zeros(G + 1, dtype=np.int64)
    gen_ms = np.zeros(G + 1, dtype=np.float64)
    evals = np.zeros(G + 1, dtype=np.int64)
    dp = np.zeros(max(1, diag_cap), dtype=np.float32)
    de = np.zeros(max(1, diag_cap), dtype=np.int64)
    _check(load().gapa_run_surrogate(ctx.handle, ctypes.byref(cfg), sg.handle if sg else None, _host_ptr(best_fit),
                                     _host_ptr(best), _host_ptr(traj), _host_ptr(gen_ms), _host_ptr(evals),
                                     _host_ptr(dp) if diag_cap else None, _host_ptr(de) if diag_cap else None,
                                     diag_cap))
    return {"best_fit": int(best_fit[0]), "best_set": best[: cfg.k].copy(), "traj": traj, "gen_ms": gen_ms,
            "exact_evals": evals, "diag_pred": dp[:diag_cap], "diag_exact": de[:diag_cap]}
