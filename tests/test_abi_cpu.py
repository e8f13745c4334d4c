"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(gapa_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_20980_gb300 import build as b

    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("gapa_graph_upload", "gapa_pop_init", "gapa_fitness", "gapa_generation", "gapa_run"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_2412_20980_gb300.gapa import EXPORTS

    assert sorted(EXPORTS) == declared_entry_points()


def test_version_and_error_string_without_gpu(lib):
    lib.gapa_version.restype = ctypes.c_char_p
    lib.gapa_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.gapa_version()
    assert isinstance(lib.gapa_last_error(), bytes)


def test_null_arguments_rejected_without_touching_a_device(lib):
    # every entry point validates its handle before any CUDA call
    lib.gapa_fitness.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    assert lib.gapa_fitness(None, None, 0, 0, None) == -1
    lib.gapa_sync.argtypes = [ctypes.c_void_p]
    assert lib.gapa_sync(None) == -1
    lib.gapa_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.gapa_create(None, 0, None) == -1


def test_oracle_builds_and_is_separate():
    import oracle

    path = oracle.build()
    assert os.path.exists(path)
    # the oracle shares no source with the CUDA library
    osrc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "gapa_internal" not in osrc and "gapa.h" not in osrc
    for f in glob.glob(os.path.join(ROOT, "paper_2412_20980_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            assert "import oracle" not in open(f).read(), f


def test_presets_follow_the_parameter_table():
    from paper_2412_20980_gb300 import PRESETS, preset_config, threshold

    cfg = preset_config("sixdst", 500, seed=3)
    assert (cfg.k, cfg.pop, cfg.gens) == (50, 80, 5000)
    assert cfg.pc_thr == threshold(0.5) and cfg.pm_thr == threshold(0.3)
    cfg = preset_config("cutoff", 2018)
    assert (cfg.k, cfg.pop) == (202, 80) and cfg.pc_thr == threshold(0.6) and cfg.pm_thr == threshold(0.2)
    assert preset_config("tde", 1000, gens=10).gens == 10 and PRESETS["tde"]["pop"] == 10
