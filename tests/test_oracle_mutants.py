"""The oracle's pins are sharp: plausible mistakes planted in a copy of the oracle are caught.

The same holds for the plain references of the SixDST objective and of the surrogate
(oracle/sixdst_ref.py, oracle/surrogate_ref.py).  For those, a small pytest plugin re-executes the
module's source with one mistake in it before the pin tests of that module run.

Each mutant below changes one thing in a copy of oracle/oracle.c: a dropped or wrong term, a wrong
sign or comparison, a wrong constant, or a wrong index.  The copy is compiled into a temporary
library, and the oracle's own pin tests (tests/test_oracle_fitness_pins.py and
tests/test_oracle_ga_pins.py) run against it in a subprocess.  The subprocess finds the copy
through GAPA_ORACLE_LIB.  Every mutant must make at least one pin fail.  The mistakes are planted
in the oracle, on the CPU, and nowhere else.

The build's own definitions, which no law of the paper fixes - the duplicate rule (reading R5),
the map of a Philox word to [0, n) (reading R9) and the counter layout - are pinned by the
hand-worked values of tests/golden/child_worked_examples.json; the mutants of those definitions
below (the other priority between A and B genes, another round-0 candidate, the blueprint's
lowest-position rule, a fill from the largest id, x mod n, a wrong tag or counter order) are
caught by them.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = [os.path.join(ROOT, "tests", "test_oracle_fitness_pins.py"),
        os.path.join(ROOT, "tests", "test_oracle_ga_pins.py")]

# name: (text in oracle.c, replacement)
MUTANTS = {
    "pair count C(c+1, 2) in the BFS sum":
        ("pc += (int64_t)sizes[c] * (int64_t)(sizes[c] - 1) / 2;",
         "pc += (int64_t)sizes[c] * (int64_t)(sizes[c] + 1) / 2;"),
    "BFS walks through deleted nodes":
        ("if (!dead[v] && !seen[v]) { seen[v] = 1; queue[tail++] = v; }",
         "if (!seen[v]) { seen[v] = 1; queue[tail++] = v; }"),
    "MCN keeps the smallest component":
        ("for (int64_t c = 0; c < ncomp; c++) if (sizes[c] > best) best = sizes[c];",
         "for (int64_t c = 0; c < ncomp; c++) if (best == 0 || sizes[c] < best) best = sizes[c];"),
    "Philox multiplier constant":
        ("uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
         "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;"),
    "Philox nine rounds":
        ("for (int round = 0; round < 10; round++) {",
         "for (int round = 0; round < 9; round++) {"),
    "Philox key schedule constant":
        ("k1 += 0xBB67AE85u;",
         "k1 += 0xBB67AE87u;"),
    "tournament keeps the highest fitness":
        ("if (best < 0 || fit[x] < fit[best] || (fit[x] == fit[best] && x < best)) best = x;",
         "if (best < 0 || fit[x] > fit[best] || (fit[x] == fit[best] && x < best)) best = x;"),
    "tournament ties to the higher index":
        ("if (best < 0 || fit[x] < fit[best] || (fit[x] == fit[best] && x < best)) best = x;",
         "if (best < 0 || fit[x] < fit[best] || (fit[x] == fit[best] && x > best)) best = x;"),
    "elite is the worst member":
        ("if (fit_in[x] < fit_in[elite]) elite = x;",
         "if (fit_in[x] > fit_in[elite]) elite = x;"),
    "crossover mask inverted":
        ("w->from_b[j] = draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_XOVER, 0) < pc_thr;",
         "w->from_b[j] = draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_XOVER, 0) >= pc_thr;"),
    "mutation never fires":
        ("w->mutated[j] = draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_MUT, 0) < pm_thr;",
         "w->mutated[j] = 0;"),
    "genes from B may repeat kept genes":
        ("if (!mutated[j] && from_b[j] && !w->kept.in[B[j]]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }",
         "if (!mutated[j] && from_b[j]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }"),
    "roulette weights favour high fitness":
        ("for (int32_t x = 0; x < s; x++) { acc += (mx - fit[x]) + 1; cum[x] = acc; }",
         "for (int32_t x = 0; x < s; x++) { acc += fit[x] + 1; cum[x] = acc; }"),
    "(mu+lambda) keeps the worst":
        ("if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;",
         "if (x[0] != y[0]) return x[0] > y[0] ? -1 : 1;"),
    "union-find joins through deleted nodes":
        ("if (v <= u || dead[v]) continue;",
         "if (v <= u) continue;"),
    "union-find pair count C(c, 2) as c^2 / 2":
        ("if (!dead[v] && parent[v] == v) pc += size[v] * (size[v] - 1) / 2;",
         "if (!dead[v] && parent[v] == v) pc += size[v] * size[v] / 2;"),
    "edge genes leave their edges in place":
        ("if (!gone[arc_id[e]] && !seen[v]) { seen[v] = 1; queue[tail++] = v; }",
         "if (!seen[v]) { seen[v] = 1; queue[tail++] = v; }"),
    "edge ids of reverse arcs looked up off by one":
        ("if (col[mid] < u) lo = mid + 1; else hi = mid;",
         "if (col[mid] <= u) lo = mid + 1; else hi = mid;"),
    "repair does not mark a taken candidate":
        ("if (!kept->in[c]) {\n                kept->in[c] = 1;\n                row[j] = c;",
         "if (!kept->in[c]) {\n                row[j] = c;"),
    "repair fill reuses the smallest free id":
        ("while (kept->in[next]) next++;\n        kept->in[next] = 1;",
         "while (kept->in[next]) next++;"),
    "a mutated position keeps parent A's gene":
        ("w->cand0[nh] = mutated[j] ? mutval[j] : A[j];",
         "w->cand0[nh] = A[j];"),
    "round-0 candidate of a repeated B gene is B[j]":
        ("w->cand0[nh] = mutated[j] ? mutval[j] : A[j];",
         "w->cand0[nh] = mutated[j] ? mutval[j] : B[j];"),
    "B genes win over A genes":
        ("    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && !from_b[j]) { row[j] = A[j]; w->kept.in[A[j]] = 1; }\n"
         "    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && from_b[j] && !w->kept.in[B[j]]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }",
         "    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && from_b[j]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }\n"
         "    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && !from_b[j] && !w->kept.in[A[j]]) { row[j] = A[j]; w->kept.in[A[j]] = 1; }"),
    "the lowest position keeps a repeated gene, the other parent's gene as candidate":
        ("    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && !from_b[j]) { row[j] = A[j]; w->kept.in[A[j]] = 1; }\n"
         "    for (int32_t j = 0; j < k; j++)\n"
         "        if (!mutated[j] && from_b[j] && !w->kept.in[B[j]]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }\n"
         "    int32_t nh = 0;\n"
         "    for (int32_t j = 0; j < k; j++) {\n"
         "        if (row[j] >= 0) continue;\n"
         "        w->holes[nh] = j;\n"
         "        w->cand0[nh] = mutated[j] ? mutval[j] : A[j];",
         "    for (int32_t j = 0; j < k; j++) {\n"
         "        const int32_t v = from_b[j] ? B[j] : A[j];\n"
         "        if (!mutated[j] && !w->kept.in[v]) { row[j] = v; w->kept.in[v] = 1; }\n"
         "    }\n"
         "    int32_t nh = 0;\n"
         "    for (int32_t j = 0; j < k; j++) {\n"
         "        if (row[j] >= 0) continue;\n"
         "        w->holes[nh] = j;\n"
         "        w->cand0[nh] = mutated[j] ? mutval[j] : (from_b[j] ? A[j] : B[j]);"),
    "repair fill from the largest free id":
        ("    int32_t next = 0;\n    for (int32_t h = 0; h < nholes; h++) {\n        while (kept->in[next]) next++;",
         "    int32_t next = n - 1;\n    for (int32_t h = 0; h < nholes; h++) {\n        while (kept->in[next]) next--;"),
    "later repair rounds retry the round-0 candidate":
        ("int32_t c = r == 0 ? cand0[h] : repair_candidate(src, j, r, n);",
         "int32_t c = cand0[h];"),
    "31 repair rounds":
        ("#define REPAIR_ROUNDS 32", "#define REPAIR_ROUNDS 31"),
    "word mapped to [0, n) by x mod n":
        ("return (int32_t)(((uint64_t)x * (uint64_t)(uint32_t)n) >> 32);",
         "return (int32_t)(x % (uint32_t)n);"),
    "counter with member and gene swapped":
        ("uint32_t ctr[4] = { j, i, g, (tag << 24) | round };\n    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };\n    uint32_t out[4];\n    oracle_philox4x32_10(ctr, key, out);\n    return out[0];",
         "uint32_t ctr[4] = { i, j, g, (tag << 24) | round };\n    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };\n    uint32_t out[4];\n    oracle_philox4x32_10(ctr, key, out);\n    return out[0];"),
    "mutation candidates drawn with the repair tag":
        ("uniform_below(draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_MUTVAL, 0), n)",
         "uniform_below(draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_REPAIR, 0), n)"),
    "(mu+lambda) ties prefer children":
        ("return x[1] < y[1] ? -1 : (x[1] > y[1]);",
         "return x[1] > y[1] ? -1 : (x[1] < y[1]);"),
}


def _build(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant text not found once: {name}"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_path = tmp_path / f"{tag}.c"
    so_path = tmp_path / f"lib{tag}.so"
    c_path.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(c_path), "-o", str(so_path)],
                   check=True)
    return str(so_path)


def _pins_pass(lib):
    env = dict(os.environ, GAPA_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 0, r.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    libs = {name: _build(name, tmp_path) for name in MUTANTS}
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(libs, ex.map(_pins_pass, libs.values())))
    survivors = [name for name, (ok, _) in results.items() if ok]
    assert not survivors, f"mistakes no pin catches: {survivors}"


def test_unmutated_copy_passes_the_pins(tmp_path):
    """The harness itself: the oracle compiled the same way from the unchanged source passes."""
    so_path = tmp_path / "liboracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", SRC, "-o", str(so_path)], check=True)
    ok, out = _pins_pass(str(so_path))
    assert ok, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_text_present(name):
    assert open(SRC).read().count(MUTANTS[name][0]) == 1, name


# name: (reference module, text in its source, replacement, pin file)
PY_MUTANTS = {
    "SixDST without the identity": (
        "oracle.sixdst_ref", "base = np.minimum(a + np.eye(n, dtype=np.int64), 1).astype(np.float64)",
        "base = np.minimum(a, 1).astype(np.float64)", "test_oracle_sixdst_pins.py"),
    "SixDST one product short": (
        "oracle.sixdst_ref", "for _ in range(hops - 1):", "for _ in range(hops - 2):", "test_oracle_sixdst_pins.py"),
    "SixDST without the normalisation": (
        "oracle.sixdst_ref", "m = np.minimum(m @ base, 1.0)", "m = m @ base", "test_oracle_sixdst_pins.py"),
    "SixDST PC counts each node with itself": (
        "oracle.sixdst_ref", "return int((rows.sum() - live.sum()) // 2)", "return int(rows.sum() // 2)",
        "test_oracle_sixdst_pins.py"),
    "SixDST keeps arcs into deleted nodes": (
        "oracle.sixdst_ref", "keep = live[src] & live[col]", "keep = live[src]", "test_oracle_sixdst_pins.py"),
    "surrogate ReLU mask of the wrong layer": (
        "oracle.surrogate_ref", 'dz2 = np.outer(dy, params["w3"]) * (c["z2"] > 0)',
        'dz2 = np.outer(dy, params["w3"]) * (c["z1"] > 0)', "test_oracle_surrogate_pins.py"),
    "surrogate b1 gradient from the second layer": (
        "oracle.surrogate_ref", 'g["b1"] = dz1.sum(axis=0)', 'g["b1"] = dz2.sum(axis=0)',
        "test_oracle_surrogate_pins.py"),
    "surrogate embedding gradient without 1/sqrt(k)": (
        "oracle.surrogate_ref", "np.add.at(gE, pop[b], dx[b, :EMB] / np.sqrt(k))", "np.add.at(gE, pop[b], dx[b, :EMB])",
        "test_oracle_surrogate_pins.py"),
    "surrogate loss gradient not averaged": (
        "oracle.surrogate_ref", "dy = 2.0 * (y - t) / B", "dy = 2.0 * (y - t)", "test_oracle_surrogate_pins.py"),
    "AdamW without bias correction": (
        "oracle.surrogate_ref", "mh = m / (1 - b1 ** tau)", "mh = m", "test_oracle_surrogate_pins.py"),
    "AdamW decay outside the learning rate": (
        "oracle.surrogate_ref", "p -= lr * (mh / (np.sqrt(vh) + eps) + wd * p)",
        "p -= lr * mh / (np.sqrt(vh) + eps) + wd * p", "test_oracle_surrogate_pins.py"),
    "residual r1 counts two live neighbours": (
        "oracle.surrogate_ref", "r1 = int(np.count_nonzero(touched & (live_nb == 1)))",
        "r1 = int(np.count_nonzero(touched & (live_nb == 2)))", "test_oracle_surrogate_pins.py"),
    "standardised counts without the floor at 1": (
        "oracle.surrogate_ref", "sd = max(np.sqrt(max(var, 0.0)), 1.0)", "sd = max(np.sqrt(max(var, 0.0)), 1e-12)",
        "test_oracle_surrogate_pins.py"),
    "stored variant masks dz1 with the second layer": (
        "oracle.surrogate_ref", "dz1 = rnd((dz2 @ W2.T) * (z1 > 0))", "dz1 = rnd((dz2 @ W2.T) * (z2 > 0))",
        "test_oracle_surrogate_pins.py"),
    "stored variant's loss gradient not averaged": (
        "oracle.surrogate_ref", "dy = 2.0 * (y - t) / y.shape[0]", "dy = 2.0 * (y - t)", "test_oracle_surrogate_pins.py"),
    "BF16 rounding truncates": (
        "oracle.surrogate_ref", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = (u >> 16) << 16",
        "test_oracle_surrogate_pins.py"),
    "degree feature: mean instead of max": (
        "oracle.surrogate_ref", "x[i, 65] = qi.max()", "x[i, 65] = qi.mean()", "test_oracle_surrogate_pins.py"),
}

PLUGIN = """
import importlib, inspect, os


def pytest_configure(config):
    mod = importlib.import_module(os.environ["GAPA_MUTANT_MODULE"])
    src = inspect.getsource(mod)
    old, new = os.environ["GAPA_MUTANT_OLD"], os.environ["GAPA_MUTANT_NEW"]
    assert src.count(old) == 1, "mutant text not found once"
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
"""


def _py_pins_pass(tmp_path, module, old, new, pin_file):
    (tmp_path / "gapa_mutant_plugin.py").write_text(PLUGIN)
    env = dict(os.environ, GAPA_MUTANT_MODULE=module, GAPA_MUTANT_OLD=old, GAPA_MUTANT_NEW=new,
               PYTHONPATH=os.pathsep.join([ROOT, str(tmp_path)] + [p for p in [os.environ.get("PYTHONPATH")] if p]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-p",
                        "gapa_mutant_plugin", os.path.join(ROOT, "tests", pin_file)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def test_every_planted_reference_mistake_fails_a_pin(tmp_path):
    for name, (module, old, new, _) in PY_MUTANTS.items():
        src = open(os.path.join(ROOT, *module.split(".")) + ".py").read()
        assert src.count(old) == 1, name
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(PY_MUTANTS, ex.map(lambda m: _py_pins_pass(tmp_path, *m), PY_MUTANTS.values())))
    survivors = [name for name, (ok, _) in results.items() if ok]
    assert not survivors, f"mistakes no pin catches: {survivors}"


@pytest.mark.parametrize("module,pin_file", [("oracle.sixdst_ref", "test_oracle_sixdst_pins.py"),
                                             ("oracle.surrogate_ref", "test_oracle_surrogate_pins.py")])
def test_reference_plugin_without_a_mistake_passes(tmp_path, module, pin_file):
    """The plugin itself: re-executing the unchanged source leaves the pins passing."""
    ok, out = _py_pins_pass(tmp_path, module, "import numpy as np", "import numpy as np", pin_file)
    assert ok, out
