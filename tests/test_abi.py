"""CPU checks of the boundary: the library builds, loads and exports every
function include/sky.h declares; the oracle and the CUDA path share no code."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"SKY_API\s+[\w\s\*]+?\b(sky_\w+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for want in ("sky_build_grid", "sky_prune_cells", "sky_skyline", "sky_grid_stats",
                 "sky_grid_destroy", "sky_status_string", "sky_last_error"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2107_09993_b300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.sky_status_string.restype = ctypes.c_char_p
    assert lib.sky_status_string(0) == b"ok"
    lib.sky_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sky_version()


def test_invalid_arguments_rejected_without_device():
    import paper_2107_09993_b300 as sky
    lib = sky.load()
    cnt = ctypes.c_int64(0)
    # d = 0 and d = 17 are rejected before any device work
    for d in (0, 17):
        st = lib.sky_skyline(None, 10, d, max(d, 1), None, None, 0, ctypes.byref(cnt), None)
        assert st == 1
        assert b"d =" in lib.sky_last_error()
    st = lib.sky_skyline(None, 10, 3, 2, None, None, 0, ctypes.byref(cnt), None)
    assert st == 1


def test_oracle_and_cuda_path_share_no_code():
    csrc = glob.glob(os.path.join(ROOT, "paper_2107_09993_b300", "**", "*"), recursive=True)
    for f in csrc:
        if f.endswith((".cu", ".cuh", ".h", ".py")):
            txt = open(f).read()
            assert "oracle" not in re.findall(r"(?:#include|import|from)\s+[\"<]?(\w+)", txt), f
            assert "sky_oracle" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".c", ".py")):
            txt = open(f).read()
            assert "paper_2107_09993_b300" not in txt, f
            assert "sky_common" not in txt and "sky.h" not in txt, f
