#!/usr/bin/env python
"""Benchmark of the batched critical-node-detection hot path on GB300.

Default workload "throughput" (one step = one GA generation on each of two graphs):
  Barabasi-Albert n=20000, m=4 (79,984 edges) and Holme-Kim n=20000, m=4,
  p=0.3 (79,984 edges); k = 1000 deleted nodes (5% of n); population s = 1024;
  tournament 2, uniform crossover pc = 0.8, per-gene mutation pm = 0.02,
  elitism 1, Philox seed = rank.  Each generation runs elitism, selection,
  crossover, mutation, duplicate repair and the exact fitness (pairwise
  connectivity) of the s-1 children, all in libgapa.so's kernels.
  Metric: exact CND fitness evaluations per second (whole job), with the
  generations per second beside it.
Other workloads (for the design notes, not the headline line):
  "large": one GA generation on R-MAT scale 20 (2^24 edges), k = 10000, s = 256;
  "small": one whole run (init + 100 generations, CUDA-graph replay) on
           BA n=1000, m=3, k = 50, s = 100; metric GA generations per second;
  "batched": 64 independent instances advanced by one batched run;
  "sixdst": one GA generation under the SixDST objective (Eqs. 14-17: N = 6
           hops, dense 0/1 reachability products on the tensor cores) on an
           Erdos-Renyi n = 2018, E = 2705 graph (the size of the paper's
           Yeast1), the paper's SixDST parameters (population 80, pc = 0.5,
           pm = 0.3, k = 10 % of n);
  "surrogate": (mu+lambda) GA on BA n=100000, m=3, k = 2000, mu = 512,
           lambda = 2048, 300 generations, plain (every child exact) against
           surrogate-screened (top 256 children exact); metric: the plain
           run's time to its final best over the screened run's time to reach
           that same value (the screened run may take up to 600 generations);
           the 1.01 x tolerance is reported beside it.

The default line (throughput workload, one GPU) also carries, under "workloads", each of the
other workloads timed in the same run with a short step count of its own: "small" (whole runs
through gapa_run), "large", "batched", "sixdst" and "surrogate" (screening the top 25 % of the
children, with 12.5 % beside it).  Rooflines of graphs that fit in L2 are graded against the L2
read bandwidth measured in the run (the library's probe), with the HBM-denominated figure beside
it; larger graphs against the measured HBM copy bandwidth.

``--impl reference`` times the CPU oracle (plain C, OpenMP over members) on a
bounded sample of the same workload.  Under torchrun (N > 1) the default mode
is the member split of Section III-D: one population per graph, every rank
runs the operators and evaluates its contiguous slice of the children, and the
int64 fitness is all-gathered over NCCL on the context's stream (strong
scaling); ``--mode independent`` gives every rank its own populations instead
(weak scaling, no collective on the data path).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PC, PM, TOURN = 0.8, 0.02, 2
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    "throughput": dict(k=1000, pop=1024, gens=1, metric="exact CND fitness evals/s", unit="evals/s",
                       desc="GA generation step on BA(n=20000,m=4) + HK(n=20000,m=4,p=0.3), k=1000, s=1024, "
                            "tournament 2, pc=0.8, pm=0.02, elitism 1",
                       graphs=["ba_n20000_m4_seed1 (E=79984)", "hk_n20000_m4_p0.3_seed1 (E=79984)"]),
    "large": dict(k=10000, pop=256, gens=1, metric="exact CND fitness evals/s", unit="evals/s",
                  desc="GA generation step on R-MAT scale 20 (2^20 nodes, 2^24 edges, a=0.57 b=0.19 c=0.19), "
                       "k=10000, s=256, tournament 2, pc=0.8, pm=0.02, elitism 1",
                  graphs=["rmat_s20_e16777216_seed1"]),
    "batched": dict(k=0, pop=0, gens=200, metric="exact CND fitness evals/s (aggregate)", unit="evals/s",
                    desc="64 independent GA instances, BA graphs with n log-uniform in [500, 50000], m in 2..5, "
                         "k = round(0.05 n), populations from {32,64,128,256,512}, 200 generations each, "
                         "one batched run per step (CUDA-graph replay, persistent fitness kernel, autotuned teams)",
                    graphs=["64 BA instances (synth.batched_instances, seed 0)"]),
    "surrogate": dict(k=2000, pop=512, lam=2048, screens=(512, 256), gens=300,
                      metric="surrogate vs plain GA time-to-target speedup", unit="x",
                      desc="(mu+lambda) GA on BA(n=100000,m=3), k=2000, mu=512, lambda=2048 children per generation, "
                           "tournament 2, pc=0.8, pm=0.02, 300 generations; one step = one GA seed "
                           "(1000 rank + step) run plain (all 2048 children exact) and surrogate-screened: the 512 "
                           "lowest-scored children exact (the top 25 %), and beside it the 256 lowest-scored "
                           "(12.5 %), after 3 warm-up generations; 2 AdamW steps of 256 rows per generation, lr 1e-3, "
                           "on a 16384-row replay ring; targets z-scored over the ring; value = median over the steps "
                           "of the 25 % setting's speedup to the plain run's final best PC",
                      graphs=["ba_n100000_m3_seed1 (E=299991)"]),
    "sixdst": dict(k=202, pop=80, gens=1, metric="SixDST fitness evals/s", unit="evals/s",
                   desc="GA generation step under the SixDST objective (N = 6 hops) on ER(n=2018,E=2705), k=202, "
                        "s=80, tournament 2, pc=0.5, pm=0.3, elitism 1",
                   graphs=["er_n2018_e2705_seed1"]),
    "small": dict(k=50, pop=100, gens=100, metric="GA gens/s", unit="gens/s",
                  desc="whole GA run: init + 100 generations on BA(n=1000,m=3), k=50, s=100, tournament 2, "
                       "pc=0.8, pm=0.02, elitism 1, Philox seed 0",
                  graphs=["ba_n1000_m3_seed1 (E=2991)"]),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def batched_specs():
    import synth

    return synth.batched_instances(64, seed=0)


def graphs(workload: str):
    import synth

    if workload == "batched":
        return [synth.ba_graph(d["n"], d["m"], d["graph_seed"]) for d in batched_specs()]
    if workload == "large":
        return [synth.rmat_graph(RMAT_SCALE[0], 16 << RMAT_SCALE[0], seed=1)]
    if workload == "small":
        return [synth.ba_graph(1000, 3, 1)]
    if workload == "surrogate":
        return [synth.ba_graph(100000, 3, 1)]
    if workload == "sixdst":
        return [synth.er_graph(2018, 2705, 1)]
    return [synth.ba_graph(20000, 4, 1), synth.hk_graph(20000, 4, 0.3, 1)]


# R-MAT scale of the large workload (20; smaller only for profiling captures, --rmat-scale):
# 16 edges per node, k = 10000 scaled with the node count
RMAT_SCALE = [20]


def large_k() -> int:
    return max(1, round(10000 * 2.0 ** (RMAT_SCALE[0] - 20)))


def bytes_per_eval(n: int, num_edges: int, k: int) -> int:
    """Algorithmic bytes of one exact evaluation: row pointers, each undirected
    edge once, the deletion bitmap, the genes and the int64 result."""
    return 4 * (n + 1) + 4 * num_edges + (n + 7) // 8 + 4 * k + 8


_L2_PEAK = {}


def l2_read_peak(ctx) -> float:
    """L2 read bandwidth (GB/s) measured once per process by the library's probe: 16-byte loads
    over a 64 MB buffer (L2-resident), fastest of 10 passes."""
    if "v" not in _L2_PEAK:
        _L2_PEAK["v"] = float(ctx.read_bandwidth(64 << 20, 10))
    return _L2_PEAK["v"]


L2_PEAK_SOURCE = ("measured here: gapa_read_bandwidth, 16-byte loads over a 64 MB buffer (L2-resident), "
                  "fastest of 10 passes")


def memory_roofline(achieved: float, l2_resident: bool, ctx, **extra) -> dict:
    """Roofline of a memory-bound fitness phase.  Graphs that fit in L2 are graded against the
    measured L2 read bandwidth, with the HBM-denominated fraction beside it; larger graphs against
    the measured HBM copy bandwidth."""
    hbm, hbm_src = measured_peaks()
    hbm_part = {"peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
    if l2_resident:
        l2 = l2_read_peak(ctx)
        r = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
             "peak_source": L2_PEAK_SOURCE, "hbm": hbm_part}
    else:
        r = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
             "peak_source": hbm_part["peak_source"]}
    r.update(extra)
    return r


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# sources the fitness kernels of each workload are compiled from: the shared-memory kernels
# (fitness.cu and its headers) and, for graphs whose labels exceed shared memory, the sparse
# kernel (fitness_sparse.cu, dispatched from fitness.cu)
TRAFFIC_SOURCES = {
    "large": ("fitness.cu", "fitness_sparse.cu", "tree16.cuh", "gapa_internal.cuh"),
    "surrogate": ("fitness.cu", "fitness_sparse.cu", "tree16.cuh", "gapa_internal.cuh"),
}
DEFAULT_TRAFFIC_SOURCES = ("fitness.cu", "tree16.cuh", "gapa_internal.cuh")


KERNEL_TEXT = {
    ("throughput", "auto"): "fitness phase: local_order_kernel + cc_smem_kernel<4> (cut-local TREE, two forests, "
                            "estimates written by the operator kernel)",
    ("small", "auto"): "cc_smem_kernel (full TREE pipeline, shared-memory labels; n <= 2048)",
    ("large", "auto"): "cc_sparse_kernel<int> (sparse: re-picked tops, hop chains, sampled terminal links, listed "
                       "pieces only; one persistent CTA per member)",
    ("large", "tree"): "ig_* kernels (interleaved global labels, 8 members per 32-byte sector)",
    ("throughput", "sparse"): "cc_sparse_kernel<unsigned short> (sparse kernel forced on a shared-memory graph)",
    ("large", "sparse"): "cc_sparse_kernel<int>",
}


def measured_traffic_fraction(traffic: float, avg_launch_s: float) -> dict:
    """DRAM bytes that ncu counted per fitness phase over the phase's duration, against the measured HBM
    copy bandwidth: the graded figure where the algorithmic bytes (a full CSR pass per member)
    overstate what a kernel that reads only the disturbed part of the graph moves."""
    hbm, src = measured_peaks()
    ach = traffic / avg_launch_s / 1e9
    return {"achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum per phase (profiles/fitness_traffic.json) "
                     f"/ CUDA-event phase time; peak {src} HBM copy bandwidth"}


def kernel_source_hash(workload: str) -> str:
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES.get(workload, DEFAULT_TRAFFIC_SOURCES):
        h.update(open(os.path.join(ROOT, "paper_2412_20980_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str):
    """dram read+write bytes per launch of the fitness kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "fitness_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(workload)
    if not d or d.get("source_hash") != kernel_source_hash(workload):
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.4)
        except Exception as e:  # no nvidia-smi: report clocks as unknown
            log("clock sampler unavailable:", e)
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 9]
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].strip() == "Active"})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(wl: str, pop=None):
    w = WORKLOADS[wl]
    pop = pop or w["pop"]
    cfg = {"workload": w["desc"], "graphs": w["graphs"], "k": w["k"], "pop": pop,
           "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
           "parallelism": "dp (independent populations per rank)"}
    if wl == "small":
        cfg["gens_per_step"] = w["gens"]
    else:
        cfg["evals_per_step"] = len(w["graphs"]) * (pop - 1)
    return cfg


# ----------------------------------------------------------------------------
# CPU oracle: baseline and reference arm
# ----------------------------------------------------------------------------
def oracle_step_fn(wl: str, gs, s_ref: int):
    """One step of the workload run by the oracle on a population of s_ref."""
    import oracle

    w = WORKLOADS[wl]
    pc_thr, pm_thr = oracle.thresholds(PC, PM)
    nt = oracle.max_threads()
    if wl == "sixdst":  # the dense reference on the members of the initial population (the evaluations dominate)
        from oracle import sixdst_ref

        pop0 = oracle.pop_init(gs[0].n, w["k"], s_ref, 0)

        def step(t):
            sixdst_ref.fitness(gs[0].row_ptr, gs[0].col, pop0[: s_ref - 1])
            return s_ref - 1
        return step, nt
    if wl == "small":
        def step(t):
            oracle.run(gs[0].row_ptr, gs[0].col, k=w["k"], pop=s_ref, gens=w["gens"], tourn=TOURN, pc_thr=pc_thr,
                       pm_thr=pm_thr, seed=0, nthreads=nt)
            return w["gens"]
        return step, nt
    pops = [oracle.pop_init(g.n, w["k"], s_ref, 0) for g in gs]
    fits = [oracle.fitness(g.row_ptr, g.col, p, nthreads=nt) for g, p in zip(gs, pops)]

    def step(t):
        for j, g in enumerate(gs):
            pops[j], fits[j] = oracle.generation(g.row_ptr, g.col, pops[j], fits[j], t + 1, tourn=TOURN,
                                                 pc_thr=pc_thr, pm_thr=pm_thr, seed=0, nthreads=nt)
        return len(gs) * (s_ref - 1)
    return step, nt


def sample_population(wl: str, gs, seconds: float) -> int:
    """Largest population (<= the workload's) whose oracle step fits the time budget."""
    import oracle

    w = WORKLOADS[wl]
    if wl == "small":
        return w["pop"]
    if wl == "sixdst":  # about 0.6 s per dense evaluation
        return max(2, min(w["pop"], int(seconds / 0.6) + 1))
    rows = min(4, w["pop"])
    pop = oracle.pop_init(gs[0].n, w["k"], rows, 0)
    t0 = time.perf_counter()
    for g in gs:
        oracle.fitness(g.row_ptr, g.col, pop, nthreads=1)
    per_member = (time.perf_counter() - t0) / rows / max(1, oracle.max_threads())
    s = int(seconds / max(per_member, 1e-9))
    return max(8, min(w["pop"], s))


def cpu_baseline(wl: str, gs, seconds: float) -> dict:
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    s_ref = sample_population(wl, gs, seconds / 2)
    step, nt = oracle_step_fn(wl, gs, s_ref)
    t0 = time.perf_counter()
    units, steps = 0, 0
    while True:
        units += step(steps)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or (wl == "large" and steps >= 1):
            break
    w = WORKLOADS[wl]
    return {"value": units / el, "unit": w["unit"], "cores": nt, "kind": "oracle",
            "sample": f"{steps} oracle steps of the workload with population {s_ref} (of {w['pop']}): "
                      f"{units} {'generations' if wl == 'small' else 'evals'} in {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    wl = args.workload
    w = WORKLOADS[wl]
    gs = graphs(wl)
    budget = 150.0
    s_ref = sample_population(wl, gs, budget / max(1, args.steps + args.warmup))
    step, nt = oracle_step_fn(wl, gs, s_ref)
    for t in range(args.warmup):
        step(t)
    t0 = time.perf_counter()
    units = 0
    for t in range(args.steps):
        units += step(args.warmup + t)
    el = time.perf_counter() - t0
    v = units / el
    sample = (f"oracle, population {s_ref} (of {w['pop']}): {args.steps} steps = {units} "
              f"{'generations' if wl == 'small' else 'evals'} in {el:.1f} s")
    line = {"impl": "reference", "metric": w["metric"], "value": v, "unit": w["unit"], "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(wl, s_ref),
            "cpu_baseline": {"value": v, "unit": w["unit"], "cores": nt, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": w["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
class Env:
    """Process-level state: the process group (or None), world size, ranks and device."""

    def __init__(self, dist, ws, rank, local, dev):
        self.dist, self.ws, self.rank, self.local, self.dev = dist, ws, rank, local, dev


def setup() -> Env:
    import torch

    from paper_2412_20980_gb300 import build as b

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        b.build()
    if dist is not None:
        dist.barrier()
    return Env(dist, ws, rank, local, dev)


def set_kernel(ctx, args):
    from paper_2412_20980_gb300 import gapa as gp

    choice = getattr(args, "fitness_kernel", "auto")
    if choice != "auto":
        ctx.set_fitness_kernel({"tree_local": gp.FITNESS_TREE_LOCAL, "tree": gp.FITNESS_TREE,
                                "piece": gp.FITNESS_PIECE, "sparse": gp.FITNESS_SPARSE}[choice])


def run_workload(args, env: Env):
    """One workload's JSON line (rank 0) or None (other ranks)."""
    gs = graphs(args.workload)
    if args.workload == "batched":
        return run_batched(args, gs, env.dist, env.ws, env.rank, env.local, env.dev)
    if args.workload == "surrogate":
        return run_surrogate_bench(args, gs, env.dist, env.ws, env.rank, env.local, env.dev)
    return run_gapa(args, env, gs)


def run_gapa(args, env: Env, gs):
    import torch

    from paper_2412_20980_gb300 import Context, make_config
    from paper_2412_20980_gb300 import dist as gd

    wl = args.workload
    w = WORKLOADS[wl]
    dist, ws, rank, local, dev = env.dist, env.ws, env.rank, env.local, env.dev
    # member split (Section III-D, SM mode): one population per graph, every rank runs the
    # operators and evaluates its slice of the children, fitness all-gathered; otherwise every
    # rank evolves its own populations
    split = args.mode == "split" and ws > 1 and wl in ("throughput", "large")
    k, pop = (large_k() if wl == "large" else w["k"]), w["pop"]
    pc, pm = (0.5, 0.3) if wl == "sixdst" else (PC, PM)
    seed = 0 if split else gd.rank_seed(0, rank)
    cfg = make_config(k=k, pop=pop, gens=w["gens"], tourn=TOURN, pc=pc, pm=pm, seed=seed)
    ctxs, state = [], []
    for g in gs:
        c = Context(local)
        set_kernel(c, args)
        c.graph_upload(g.row_ptr, g.col)
        if wl == "sixdst":
            from paper_2412_20980_gb300.gapa import OBJECTIVE_SIXDST_PC

            c.set_objective(OBJECTIVE_SIXDST_PC)
        pa = c.pop_init(cfg)
        fa = c.fitness(pa)
        state.append([pa, fa, torch.empty_like(pa), torch.empty_like(fa)])
        ctxs.append(c)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    if wl == "small":
        def step(t):
            for c in ctxs:
                c.run(cfg)  # synchronous: init + gens generations, best set copied to the host
            return len(ctxs) * w["gens"]
    elif split:
        def step(t):
            for c, st in zip(ctxs, state):
                gd.sharded_generation(c, cfg, t + 1, st[0], st[1], st[2], st[3])
                st[0], st[2] = st[2], st[0]
                st[1], st[3] = st[3], st[1]
            return len(ctxs) * (pop - 1)
    else:
        def step(t):
            for c, st in zip(ctxs, state):
                c.generation(cfg, t + 1, st[0], st[1], st[2], st[3])
                st[0], st[2] = st[2], st[0]
                st[1], st[3] = st[3], st[1]
            return len(ctxs) * (pop - 1)

    for t in range(args.warmup):
        step(t)
    torch.cuda.synchronize()
    # --- timed region: device time per step, L2 flushed between steps ---
    sampler = ClockSampler(local)
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for c in ctxs:
        c.profile_begin()
    units = 0
    for t in range(args.steps):
        flush.fill_(t & 0xFF)
        starts[t].record()
        units += step(args.warmup + t)
        ends[t].record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    profs = [c.profile_end() for c in ctxs]
    clocks = sampler.stop()
    total_ms = gd.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), device=dev)
    for c in ctxs:
        c.sync()
    # the split evaluates one population per graph on all ranks together; independent populations
    # add up over the ranks
    job_units = units if split else units * ws
    value = job_units / (total_ms / 1000.0)

    # --- dominant kernel: the fitness launches inside the timed region ---
    fit_ms = sum(p["fitness_ms"] for p in profs)
    fit_launches = sum(p["fitness_launches"] for p in profs)
    fit_calls = sum(p["fitness_calls"] for p in profs)
    fit_evals = sum(p["evals"] for p in profs)
    roofline = None
    if wl == "small":
        # whole runs replay CUDA graphs (the profiler sees only the first fitness launch); a
        # 1000-node graph is launch- and latency-bound, graded by generations per second
        fit_launches = 0
    if fit_launches and wl == "sixdst":
        # tensor-bound: 3 dense products of n x n 0/1 matrices per evaluation ((A+I)^2, ^4, ^6)
        flop = 3 * 2.0 * float(gs[0].n) ** 3
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        peak = 2.0 * float(d["bf16_tflops"])
        achieved = flop * fit_evals / (fit_ms / 1000.0) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None,
                    "kernel": "sdst_gemm_t7_kernel (tcgen05.mma kind::f8f6f4 E4M3, operands loaded by "
                              "cp.async.bulk.tensor in 128-byte swizzled boxes, producer and MMA threads split, "
                              "256 x 256 tiles as two M = 128, N = 256 products, FP32 accumulators in TMEM)",
                    "flop_per_eval": flop, "evals": fit_evals, "fitness_ms": fit_ms,
                    "peak_source": "measured bf16 burst (MEASURED_PEAKS.json bf16_tflops) x 2, the FP8/BF16 nominal "
                                   "ratio" if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else
                                   "fallback 1.9 PFLOP/s bf16 x 2",
                    "fitness_share_of_step": fit_ms / max(1e-9, total_ms)}
    elif fit_launches:
        beval = bytes_per_eval(gs[0].n, gs[0].num_edges, k)
        # per fitness phase (one per graph and generation): its kernels together, timed on the
        # launching stream around the phase
        avg_launch_s = fit_ms / 1000.0 / fit_calls
        achieved = beval * (fit_evals / fit_calls) / avg_launch_s / 1e9
        traffic = ncu_traffic(wl) if RMAT_SCALE[0] == 20 else None
        roofline = memory_roofline(
            achieved, wl in ("throughput", "small"), ctxs[0],
            traffic=traffic,
            kernel=KERNEL_TEXT.get((wl, getattr(args, "fitness_kernel", "auto")), "fitness phase"),
            kernels_per_phase=fit_launches / fit_calls, bytes_per_eval=beval,
            evals_per_launch=fit_evals / fit_calls, avg_launch_ms=avg_launch_s * 1000,
            fitness_share_of_step=fit_ms / max(1e-9, total_ms))
        if traffic:
            roofline["measured"] = measured_traffic_fraction(traffic, avg_launch_s)

    # --- end to end through the C ABI with pinned host buffers ---
    e2e = None
    if not args.no_e2e and wl != "small":
        hp, pinned = [], []
        for c, st in zip(ctxs, state):
            ts = [st[0].cpu().pin_memory(), st[1].cpu().pin_memory(),
                  torch.empty(st[0].shape, dtype=torch.int32).pin_memory(),
                  torch.empty(st[1].shape, dtype=torch.int64).pin_memory()]
            pinned.append(ts)  # keeps the page-locked buffers alive
            hp.append([t.numpy() for t in ts])
        e2e_steps = max(3, min(args.steps, 50))
        torch.cuda.synchronize()
        el = 0.0
        for t in range(e2e_steps):
            flush.fill_(t & 0xFF)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            for c, h, ts, st in zip(ctxs, hp, pinned, state):
                if split:  # host population in, split generation, population and fitness out
                    st[0].copy_(ts[0], non_blocking=True)
                    st[1].copy_(ts[1], non_blocking=True)
                    gd.sharded_generation(c, cfg, 10_000 + t, st[0], st[1], st[2], st[3])
                    ts[2].copy_(st[2], non_blocking=True)
                    ts[3].copy_(st[3], non_blocking=True)
                    torch.cuda.current_stream().synchronize()
                else:
                    c.generation_host(cfg, 10_000 + t, h[0], h[1], h[2], h[3])
                ts[0], ts[2] = ts[2], ts[0]
                ts[1], ts[3] = ts[3], ts[1]
                h[0], h[2] = h[2], h[0]
                h[1], h[3] = h[3], h[1]
            el += time.perf_counter() - t0
        el = gd.max_over_ranks(el, device=dev)
        per = len(gs) * (pop * k * 4 + pop * 8)
        e2e = {"value": len(gs) * (pop - 1) * e2e_steps * (1 if split else ws) / el, "unit": "evals/s",
               "h2d_bytes_per_step": per, "d2h_bytes_per_step": per, "steps": e2e_steps,
               "api": ("Context + dist.sharded_generation with pinned host population and fitness copied in and out"
                       if split else "gapa_generation_host (pinned host population and fitness in and out)")}

    if dist is not None:
        dist.barrier()
    if rank != 0:
        for c in ctxs:
            c.close()
        return None
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, gs, args.cpu_seconds)
    config = workload_config(wl)
    if split:
        config["parallelism"] = (f"member split over {ws} ranks (one population per graph; operators on every "
                                 "rank, fitness by contiguous slices, int64 fitness all-gathered over NCCL)")
    line = {"metric": w["metric"], "value": value, "unit": w["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config}
    if wl == "small":
        line["evals_per_s"] = units * (pop - 1) * ws / (total_ms / 1000.0)
    else:
        line["gens_per_s"] = args.steps * len(gs) * (1 if split else ws) / (total_ms / 1000.0)
    line.update({"roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                 "gpu_launches": int(sum(p["fitness_launches"] + p["operator_launches"] for p in profs)),
                 "clocks": clocks})
    for c in ctxs:
        c.close()
    return line


def run_batched(args, gs, dist, ws, rank, local, dev):
    """64 instances per step: one gapa_batch_run of 200 generations (all on the device)."""
    import torch

    from paper_2412_20980_gb300 import Batch, Context, make_config

    w = WORKLOADS["batched"]
    specs = batched_specs()
    ctxs, cfgs = [], []
    for d, g in zip(specs, gs):
        c = Context(local)
        c.graph_upload(g.row_ptr, g.col)
        ctxs.append(c)
        cfgs.append(make_config(k=d["k"], pop=d["pop"], tourn=TOURN, pc=PC, pm=PM, seed=1000 * rank + d["index"]))
    bt = Batch(ctxs, cfgs)
    t0 = time.perf_counter()
    bt.autotune(os.path.join(ROOT, ".cache", "batch_teams.json") if os.path.isdir(os.path.join(ROOT, ".cache"))
                else None)
    tune_s = time.perf_counter() - t0
    gens = args.gens or w["gens"]
    evals_per_run = sum(d["pop"] + (d["pop"] - 1) * gens for d in specs)
    # algorithmic bytes of every exact evaluation of a run, instance by instance
    bytes_per_run = sum((d["pop"] + (d["pop"] - 1) * gens) * bytes_per_eval(g.n, g.num_edges, d["k"])
                        for d, g in zip(specs, gs))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        bt.run(gens)
    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall, dev_ms = 0.0, 0.0
    for t in range(args.steps):
        flush.fill_(t & 0xFF)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record()  # the batch runs on the first context's stream: torch's current stream
        out = bt.run(gens)  # synchronous: results are on the host when it returns
        ev1.record()
        wall += time.perf_counter() - t0
        ev1.synchronize()
        dev_ms += ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    t_max = torch.tensor([wall, dev_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    wall, dev_ms = float(t_max[0].item()), float(t_max[1].item())
    value = evals_per_run * args.steps * ws / wall
    roofline = memory_roofline(
        bytes_per_run * args.steps / (dev_ms / 1000.0) / 1e9, True, ctxs[0],
        traffic=None,
        kernel="whole batched runs (operators + fitness_batched_kernel + record, CUDA-graph replay) on the device: "
               "a lower bound on the fitness kernel's own rate",
        bytes_per_run=bytes_per_run, device_ms_per_run=dev_ms / args.steps,
        basis="sum over instances of (evaluations x 4(n+1) + 4E + ceil(n/8) + 4k + 8) per run / device time of "
              "the run")
    if rank != 0:
        bt.close()
        return None
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        import oracle

        # bounded sample: eight instances spread over the size range, 3 generations each
        order = sorted(range(len(specs)), key=lambda i: specs[i]["n"])
        idx = [order[round(q * (len(order) - 1) / 7)] for q in range(8)]
        t0 = time.perf_counter()
        units = 0
        for i in idx:
            d = specs[i]
            pc_thr, pm_thr = oracle.thresholds(PC, PM)
            oracle.run(gs[i].row_ptr, gs[i].col, k=d["k"], pop=d["pop"], gens=3, tourn=TOURN, pc_thr=pc_thr,
                       pm_thr=pm_thr, seed=d["index"], nthreads=oracle.max_threads())
            units += d["pop"] + (d["pop"] - 1) * 3
        el = time.perf_counter() - t0
        cpu = {"value": units / el, "unit": "evals/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"oracle runs of 8 instances at the size octiles, 3 generations each: {units} evals "
                         f"in {el:.1f} s"}
    line = {"metric": w["metric"], "value": value, "unit": w["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w["desc"], "instances": len(specs), "generations": gens,
                       "evals_per_step": evals_per_run, "teams": bt.teams, "autotune_s": tune_s,
                       "sum_n": sum(d["n"] for d in specs), "l2": "flushed between timed steps"},
            "gens_per_s": len(specs) * gens * args.steps * ws / wall, "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(8 * len(specs) * (gens + 2) + 4 * sum(d["k"] for d in specs)),
                    "note": "gapa_batch_run is host-synchronous: the timed wall time includes the copies of best "
                            "sets, fitness and trajectories"},
            "gpu_launches": 3 * gens * args.steps,
            "clocks": clocks, "best_fit_first8": out["best_fit"][:8].tolist()}
    bt.close()
    for c in ctxs:
        c.close()
    return line


def _spearman(a, b) -> float:
    """Spearman rank correlation (average ranks for ties)."""
    def ranks(x):
        x = np.asarray(x, dtype=np.float64)
        order = np.argsort(x, kind="stable")
        xs = x[order]
        r = np.empty(x.size)
        i = 0
        while i < x.size:
            j = i
            while j + 1 < x.size and xs[j + 1] == xs[i]:
                j += 1
            r[order[i:j + 1]] = (i + j) / 2.0
            i = j + 1
        return r
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def time_to_target(runs, G: int, lam: int):
    """Per GA seed: the plain run's device time to its final best PC, and the screened run's
    device time to reach that same value (and 1.01 x it); returns (speedups, rows)."""
    speedups, rows = [], []
    for plain, plain_wall, sur, sur_wall in runs:
        final = int(plain["traj"][-1])
        t_plain = float(plain["gen_ms"][np.nonzero(plain["traj"] == final)[0][0]])
        hit = np.nonzero(sur["traj"] <= final)[0]
        hit1 = np.nonzero(sur["traj"] <= final * 1.01)[0]
        t_sur = float(sur["gen_ms"][hit[0]]) if hit.size else None
        t_sur1 = float(sur["gen_ms"][hit1[0]]) if hit1.size else None
        speedups.append(t_plain / t_sur if t_sur else 0.0)
        rows.append({"plain_final_pc": final, "plain_initial_best_pc": int(plain["traj"][0]),
                     "surrogate_pc_at_300": int(sur["traj"][min(G, len(sur["traj"]) - 1)]),
                     "surrogate_final_pc": int(sur["traj"][-1]),
                     "plain_ms_to_final": t_plain, "surrogate_ms_to_plain_final": t_sur,
                     "surrogate_generation_at_plain_final": int(hit[0]) if hit.size else None,
                     "speedup_to_plain_final": t_plain / t_sur if t_sur else 0.0,
                     "surrogate_ms_to_1.01x": t_sur1,
                     "surrogate_generation_at_1.01x": int(hit1[0]) if hit1.size else None,
                     "speedup_to_1.01x": t_plain / t_sur1 if t_sur1 else 0.0,
                     "plain_run_ms": float(plain["gen_ms"][-1]), "surrogate_run_ms": float(sur["gen_ms"][-1]),
                     "plain_wall_s": plain_wall, "surrogate_wall_s": sur_wall,
                     "plain_exact_evals_per_s": float(plain["exact_evals"].sum() / (plain["gen_ms"][-1] / 1e3)),
                     "surrogate_exact_evals_per_s": float(sur["exact_evals"].sum() / (sur["gen_ms"][-1] / 1e3)),
                     "surrogate_children_per_s": float(lam * 2 * G / (sur["gen_ms"][-1] / 1e3))})
    return speedups, rows


def run_surrogate_bench(args, gs, dist, ws, rank, local, dev):
    """Time-to-target of the surrogate-screened GA against the plain GA (same seed, same graph)."""
    import torch

    from paper_2412_20980_gb300 import (FLAG_MU_PLUS_LAMBDA, Context, Surrogate, make_config,
                                        make_surrogate_config, run_surrogate)

    w = WORKLOADS["surrogate"]
    g = gs[0]
    G, lam = args.gens or w["gens"], w["lam"]
    ctx = Context(local)
    ctx.graph_upload(g.row_ptr, g.col)

    def config(gens, seed):
        return make_config(k=w["k"], pop=w["pop"], gens=gens, tourn=TOURN, pc=PC, pm=PM, seed=seed,
                           flags=FLAG_MU_PLUS_LAMBDA, lam=lam)

    screens = list(w["screens"])

    def scfg(diag_every=0, screened=None):
        return make_surrogate_config(screened=screened or screens[0], warmup=3, train_steps=args.sur_steps,
                                     batch=args.sur_batch,
                                     ring=16384, lr=1e-3, init_scale_emb=0.01, target_mode=0, diag_every=diag_every)

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for t in range(args.warmup):  # short runs of both kinds: module load, allocations, autotuned limits
        run_surrogate(ctx, config(5, 999), None)
        sg = Surrogate(ctx, scfg(), seed=1000 + t)
        run_surrogate(ctx, config(5, 999), sg)
        sg.close()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    runs = {sc: [] for sc in screens}
    for t in range(args.steps):  # step t: GA seed 1000 * rank + t for both arms, surrogate weights seed t
        cfg, cfg_long = config(G, 1000 * rank + t), config(2 * G, 1000 * rank + t)
        flush.fill_(t & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = run_surrogate(ctx, cfg, None)
        plain_wall = time.perf_counter() - t0
        for sc in screens:
            flush.fill_((t + 1) & 0xFF)
            sg = Surrogate(ctx, scfg(screened=sc), seed=t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sur = run_surrogate(ctx, cfg_long, sg)
            sur_wall = time.perf_counter() - t0
            sg.close()
            runs[sc].append((plain, plain_wall, sur, sur_wall))
    clocks = sampler.stop()
    # untimed: the same last runs again with CUDA events around every launch (the phase split and
    # the launch count; the events themselves cost time, so the timed runs above go without them)
    t = args.steps - 1
    for i, sc in enumerate([None] + screens):
        sg = Surrogate(ctx, scfg(screened=sc), seed=t) if sc else None
        ctx.profile_begin()
        r = run_surrogate(ctx, config(G, 1000 * rank + t) if sc is None else config(2 * G, 1000 * rank + t), sg)
        prof_r = ctx.profile_end()
        if sg:
            sg.close()
        for run in runs[sc if sc else screens[0]][t:t + 1]:
            (run[0] if sc is None else run[2])["prof"] = prof_r
        if sc is None:
            for sc2 in screens[1:]:
                runs[sc2][t][0]["prof"] = prof_r
    by_screen = {sc: time_to_target(runs[sc], G, lam) for sc in screens}
    speedups, rows = by_screen[screens[0]]
    value = float(np.median(speedups))
    tot_ms = sum(r["plain_run_ms"] + r["surrogate_run_ms"] for r in rows)
    t_max = torch.tensor([value, tot_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        t_min = t_max.clone()
        dist.all_reduce(t_min, op=dist.ReduceOp.MIN)
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        value, tot_ms = float(t_min[0].item()), float(t_max[1].item())
    all_runs = runs
    runs = runs[screens[0]]
    # untimed: a diagnostic run (surrogate quality)
    prof = runs[-1][2]["prof"]
    sg = Surrogate(ctx, scfg(diag_every=10), seed=0)
    diag = run_surrogate(ctx, config(G, 1000 * rank), sg, diag_cap=(G // 10) * lam)
    sg.close()
    rhos, relerr = [], []
    for i in range(G // 10):
        pr = diag["diag_pred"][i * lam:(i + 1) * lam].astype(np.float64)
        ex = diag["diag_exact"][i * lam:(i + 1) * lam].astype(np.float64)
        if ex.size and np.all(ex > 0):
            rhos.append(_spearman(pr, ex))
            relerr.append(float(np.median(np.abs(pr - ex) / ex)))
    if dist is not None:
        dist.barrier()
    if rank != 0:
        ctx.close()
        return None
    beval = bytes_per_eval(g.n, g.num_edges, w["k"])
    roofline = None
    if prof["fitness_calls"]:
        # the graph (1.2 M arcs) is L2-resident; per-member state in the sparse kernel's global scratch
        avg_launch_s = prof["fitness_ms"] / 1e3 / prof["fitness_calls"]
        achieved = beval * prof["evals"] / prof["fitness_calls"] / avg_launch_s / 1e9
        roofline = memory_roofline(achieved, True, ctx, traffic=ncu_traffic("surrogate"),
                                   kernel="fitness phase (screened children; cc_sparse_kernel<int>)",
                                   kernels_per_phase=prof["fitness_launches"] / prof["fitness_calls"],
                                   bytes_per_eval=beval, evals_per_launch=prof["evals"] / prof["fitness_calls"],
                                   avg_launch_ms=avg_launch_s * 1e3)
    run_ms = prof["fitness_ms"] + prof["operators_ms"] + prof["surrogate_ms"]

    def launches_of(r):
        return int(r["prof"]["fitness_launches"] + r["prof"]["operator_launches"] + r["prof"]["surrogate_launches"])

    # launches per timed step, from the profiled repeat of the last step's runs
    launches = args.steps * (launches_of(runs[-1][0]) + sum(launches_of(all_runs[sc][-1][2]) for sc in screens))
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        import oracle

        # bounded sample: oracle (mu+lambda) generations of the plain GA on the same graph
        pc_thr, pm_thr = oracle.thresholds(PC, PM)
        nt = oracle.max_threads()
        t0 = time.perf_counter()
        pop = oracle.pop_init(g.n, w["k"], w["pop"], 0)
        fit = oracle.fitness(g.row_ptr, g.col, pop, nthreads=nt)
        units, gens_done = w["pop"], 0
        while time.perf_counter() - t0 < args.cpu_seconds and gens_done < 3:
            gens_done += 1
            pop, fit = oracle.generation(g.row_ptr, g.col, pop, fit, gens_done, tourn=TOURN, pc_thr=pc_thr,
                                         pm_thr=pm_thr, seed=0, flags=oracle.FLAG_MU_PLUS_LAMBDA, lam=lam,
                                         nthreads=nt)
            units += lam
        el = time.perf_counter() - t0
        cpu = {"value": units / el, "unit": "exact evals/s", "cores": nt, "kind": "oracle",
               "sample": f"oracle plain (mu+lambda) GA on the same graph: init + {gens_done} generations = "
                         f"{units} exact evals in {el:.1f} s; the 300-generation plain run extrapolates to "
                         f"{(w['pop'] + lam * G) / (units / el):.0f} s"}
    line = {"metric": w["metric"], "value": value, "unit": w["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 fitness; bf16/fp32 surrogate",
            "data": "synthetic",
            "config": {"workload": w["desc"], "graphs": w["graphs"], "k": w["k"], "mu": w["pop"], "lambda": lam,
                       "screened": screens[0], "screened_fraction": screens[0] / lam, "generations": G,
                       "l2": "flushed before every timed run", "parallelism": "dp (independent runs per rank)",
                       "timing": "device time from CUDA events recorded by gapa_run_surrogate on its stream "
                                 "(one per generation); the phase split comes from an untimed repeat of the last "
                                 "step's runs with events around every launch"},
            "runs": rows,
            "by_screen": {str(sc): {"screened_fraction": sc / lam,
                                    "speedup_to_plain_final_median": float(np.median(by_screen[sc][0])),
                                    "speedups": by_screen[sc][0],
                                    "speedup_to_1.01x": [r["speedup_to_1.01x"] for r in by_screen[sc][1]],
                                    "surrogate_generation_at_plain_final":
                                        [r["surrogate_generation_at_plain_final"] for r in by_screen[sc][1]],
                                    "surrogate_generation_at_1.01x":
                                        [r["surrogate_generation_at_1.01x"] for r in by_screen[sc][1]]}
                          for sc in screens},
            "surrogate_quality": {"spearman_mean": float(np.mean(rhos)) if rhos else None,
                                  "spearman_min": float(np.min(rhos)) if rhos else None,
                                  "median_relative_error_mean": float(np.mean(relerr)) if relerr else None,
                                  "diagnostic_generations": len(rhos),
                                  "method": "diagnostic run (same seed) evaluating all 2048 children exactly every "
                                            "10th generation; Spearman and median |estimate - PC| / PC per "
                                            "generation"},
            "phase_split_ms": {"screened_run": {"fitness": prof["fitness_ms"], "operators": prof["operators_ms"],
                                                "surrogate": prof["surrogate_ms"], "sum": run_ms,
                                                "note": "from the profiled repeat, whose generations are launched "
                                                        "one by one (the timed runs replay steady generations from "
                                                        "CUDA graphs)"},
                               "screened_run_timed": {
                                   "total": rows[-1]["surrogate_run_ms"],
                                   "surrogate_est": rows[-1]["surrogate_run_ms"] - prof["fitness_ms"] - prof["operators_ms"],
                                   "surrogate_share_est": (rows[-1]["surrogate_run_ms"] - prof["fitness_ms"] -
                                                           prof["operators_ms"]) / rows[-1]["surrogate_run_ms"],
                                   "note": "timed run total less the profiled repeat's fitness and operator time"},
                               "plain_run": {"fitness": runs[-1][0]["prof"]["fitness_ms"],
                                             "operators": runs[-1][0]["prof"]["operators_ms"]}},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": float(min(
                        (r["plain_wall_s"] * r["plain_ms_to_final"] / r["plain_run_ms"]) /
                        (r["surrogate_wall_s"] * r["surrogate_ms_to_plain_final"] / r["surrogate_run_ms"])
                        if r["surrogate_ms_to_plain_final"] else 0.0 for r in rows)), "unit": "x",
                    "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(2 * (8 + 4 * w["k"]) + 3 * 8 * (3 * G + 2)),
                    "note": "host wall clock of each gapa_run_surrogate call (graph resident; results copied to the "
                            "host inside the call), apportioned to the target generation by the run's device-time "
                            "fraction"},
            "gpu_launches": launches,
            "clocks": clocks}
    ctx.close()
    return line


# workloads timed beside the headline in the default line: (steps, warm-up, CPU-baseline seconds)
EXTRA = {"small": (20, 3, 3.0), "large": (5, 3, 3.0), "batched": (3, 3, 3.0), "sixdst": (10, 3, 3.0),
         "surrogate": (2, 3, 3.0)}
EXTRA_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "gens_per_s", "evals_per_s", "roofline",
              "cpu_baseline", "e2e", "gpu_launches", "clocks", "by_screen", "surrogate_quality", "phase_split_ms")


def run_extra(args, env: Env) -> dict:
    """The other workloads, each timed in this same run with its own short step count."""
    out = {}
    for wl, (steps, warmup, cpu_s) in EXTRA.items():
        sub = argparse.Namespace(**vars(args))
        sub.workload, sub.steps, sub.warmup, sub.cpu_seconds = wl, steps, warmup, cpu_s
        t0 = time.perf_counter()
        line = run_workload(sub, env)
        if line is None:
            continue
        d = {key: line[key] for key in EXTRA_KEYS if key in line}
        d["config"] = line["config"].get("workload")
        d["bench_wall_s"] = time.perf_counter() - t0
        out[wl] = d
        log(f"{wl}: {line['value']:.4g} {line['unit']} ({d['bench_wall_s']:.1f} s)")
    return out


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for the throughput workload, else the workload's own count "
                         "in the default line)")
    ap.add_argument("--warmup", type=int, default=None,
                    help="untimed warm-up steps, at least 3 (default: 5 for throughput, else the workload's own)")
    ap.add_argument("--impl", choices=["gapa", "reference"], default="gapa")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="throughput")
    ap.add_argument("--mode", choices=["split", "independent"], default="split",
                    help="with several ranks: split one population by members (default) or evolve independent "
                         "populations per rank")
    ap.add_argument("--fitness-kernel", choices=["auto", "tree_local", "tree", "piece", "sparse"], default="auto",
                    help="fitness kernel of the contexts (default: the library's choice)")
    ap.add_argument("--gens", type=int, default=0,
                    help="generations per run of the batched and surrogate workloads (default: the workload's; "
                         "shorter runs are for profiling, not for the reported line)")
    ap.add_argument("--rmat-scale", type=int, default=20,
                    help="large workload: R-MAT scale (20; smaller for profiling captures: 16 edges per node, "
                         "k = 10000 scaled with the nodes)")
    ap.add_argument("--sur-steps", type=int, default=2, help="surrogate workload: AdamW steps per generation")
    ap.add_argument("--sur-batch", type=int, default=256, help="surrogate workload: rows per AdamW step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads that the default line carries under 'workloads'")
    args = ap.parse_args(argv)
    own = EXTRA.get(args.workload)
    if args.steps is None:
        args.steps = own[0] if own and args.workload != "throughput" else 200
    if args.warmup is None:
        args.warmup = own[1] if own and args.workload != "throughput" else 5
    if args.warmup < 3 and args.impl == "gapa":
        log("warm-up raised to 3 steps")
        args.warmup = 3
    return args


def main():
    args = parse_args()
    RMAT_SCALE[0] = args.rmat_scale
    if args.impl == "reference":
        return run_reference(args)
    env = setup()
    line = run_workload(args, env)
    if line is not None and args.workload == "throughput" and env.ws == 1 and not args.no_extra:
        line["workloads"] = run_extra(args, env)
    if line is not None:
        print(json.dumps(line), flush=True)
    if env.dist is not None:
        env.dist.barrier()
        env.dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
