"""Host-side checks of bench.py: the reference arm's JSON line (the oracle on the host cores), its
rank rule under several processes, the algorithmic bytes per evaluation used for the roofline, the
rule that a recorded DRAM-traffic figure is reported only while its kernel sources are the ones it
was taken on, and the step and warm-up counts each workload runs with.  No GPU is touched."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run_reference(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    """One whole 100-generation oracle run of the small workload: one JSON line with the metric,
    unit and configuration of that workload, the oracle as its CPU baseline, and an end-to-end
    figure equal to the value with no host-device bytes."""
    r = _run_reference(None, "--workload", "small", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    w = bench.WORKLOADS["small"]
    assert d["impl"] == "reference"
    assert d["metric"] == w["metric"] and d["unit"] == w["unit"]
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == w["desc"] and d["config"]["gens_per_step"] == w["gens"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == w["unit"]
    assert cb["cores"] >= 1 and "population 100" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": w["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["vs_baseline"] is None and d["data"] == "synthetic"


def test_reference_arm_other_ranks_exit_quietly():
    """Under several processes only rank 0 runs the oracle and prints; the others exit 0 with no
    output and no work."""
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--workload", "throughput",
                       "--steps", "5", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_bytes_per_eval_counts_each_input_once():
    """Row pointers, each undirected edge once (one int32 end per arc), the deletion bitmap, the
    genes and the int64 result: for the BA n = 20000, m = 4 graph (E = 79984) and k = 1000."""
    n, e, k = 20000, 79984, 1000
    want = 4 * 20001 + 4 * 79984 + 2500 + 4000 + 8
    assert bench.bytes_per_eval(n, e, k) == want == 406448
    assert bench.bytes_per_eval(1, 0, 0) == 8 + 1 + 8  # two row pointers, one bitmap byte, the result
    assert bench.bytes_per_eval(9, 0, 0) - bench.bytes_per_eval(8, 0, 0) == 4 + 1  # a new bitmap byte


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    """A traffic record is returned while the hash of its workload's kernel sources matches the one
    stored with it, and not once any of those sources changes."""
    csrc = tmp_path / "paper_2412_20980_gb300" / "csrc"
    csrc.mkdir(parents=True)
    names = set(bench.DEFAULT_TRAFFIC_SOURCES) | {f for v in bench.TRAFFIC_SOURCES.values() for f in v}
    for f in names:
        (csrc / f).write_text(f"// {f}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {wl: {"source_hash": bench.kernel_source_hash(wl), "dram_bytes_per_launch": 1000 + i}
           for i, wl in enumerate(("throughput", "large"))}
    (tmp_path / "profiles" / "fitness_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("throughput") == 1000 and bench.ncu_traffic("large") == 1001
    assert bench.ncu_traffic("sixdst") is None  # no record
    # the sparse kernel's source belongs to the large workload's kernels only
    (csrc / "fitness_sparse.cu").write_text("// changed\n")
    assert bench.ncu_traffic("throughput") == 1000 and bench.ncu_traffic("large") is None
    # a shared source invalidates both
    (csrc / "gapa_internal.cuh").write_text("// changed\n")
    assert bench.ncu_traffic("throughput") is None


@pytest.mark.parametrize("wl", sorted(bench.WORKLOADS))
def test_workload_table_is_complete(wl):
    w = bench.WORKLOADS[wl]
    for key in ("metric", "unit", "desc", "graphs"):
        assert w[key], key


def test_step_defaults_follow_the_workload():
    a = bench.parse_args([])
    assert (a.workload, a.steps, a.warmup, a.gpus) == ("throughput", 200, 5, 1)
    for wl, (steps, warmup, _) in bench.EXTRA.items():
        a = bench.parse_args(["--workload", wl])
        assert (a.steps, a.warmup) == (steps, max(warmup, 3)), wl
    a = bench.parse_args(["--workload", "surrogate", "--steps", "7", "--warmup", "1"])
    assert (a.steps, a.warmup) == (7, 3)  # never fewer than three warm-up steps


def test_every_reported_workload_warms_up_three_steps():
    assert all(warmup >= 3 for _, warmup, _ in bench.EXTRA.values())

