"""Python binding of libsky (include/sky.h): exact SkyCell skyline on one GPU.

This module only marshals arguments: torch tensors in, torch tensors out.
Every step of the skyline path runs in the CUDA kernels of libsky.so
(compiled for sm_103a by ``build.py``). There is no CPU fallback: if the
library or a CUDA device is missing, every call raises.

    import paper_2107_09993_b300 as sky
    idx = sky.skyline(points_cuda_f32)          # ascending int32 row ids

Names follow the C ABI: ``skyline`` (sky_skyline), ``skyline_host``
(sky_skyline_host), ``Grid`` (sky_build_grid / sky_prune_cells /
sky_grid_stats / sky_grid_copy_out / sky_grid_destroy).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsky.so")

SKY_OK = 0
STATUS = {
    0: "SKY_OK", 1: "SKY_ERR_INVALID_ARGUMENT", 2: "SKY_ERR_NONFINITE", 3: "SKY_ERR_CAPACITY",
    4: "SKY_ERR_OUT_OF_MEMORY", 5: "SKY_ERR_CUDA", 6: "SKY_ERR_TOO_LARGE", 7: "SKY_ERR_TIMEOUT",
    8: "SKY_ERR_NO_DEVICE",
}
GRID_CELL_KEY, GRID_OCCUPIED, GRID_DOMINATED, GRID_SURVIVORS, GRID_CELL_MAP = range(5)

_i32, _i64, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t


class SkyError(RuntimeError):
    def __init__(self, status: int, detail: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {detail}")


class Options(ctypes.Structure):
    _fields_ = [("log2_g", _i32), ("assume_unit", _i32), ("d_filter_pts", _vp),
                ("n_filter", _i32), ("tile_cfg", _i32)]


class GridStats(ctypes.Structure):
    _fields_ = [("log2_g", _i32), ("d", _i32), ("n", _i64), ("occupied_cells", _i64),
                ("surviving_cells", _i64), ("surviving_points", _i64), ("n_filter_used", _i32),
                ("error_flags", _i32)]


class RunStats(ctypes.Structure):
    _fields_ = [("n", _i64), ("d", _i32), ("log2_g", _i32), ("survivors", _i64), ("skyline", _i64),
                ("pairs", _i64), ("n_filter_used", _i32), ("kernels", _i32), ("tiles", _i64),
                ("group_scans", _i64)]


class PhaseTimes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("normalize_ms", "map_mark_ms", "prune_ms", "survivors_ms",
                                               "sort_ms", "gather_ms", "refine_ms", "emit_ms")]


_lib = None


def load():
    """Load libsky.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsky.so not built ({LIB_PATH}); run paper_2107_09993_b300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "sky_skyline": ([_vp, _i64, _i32, _i64, P(Options), _vp, _i64, P(_i64), _vp], _i32),
        "sky_skyline_host": ([_vp, _i64, _i32, _i64, P(Options), _vp, _i64, P(_i64), _vp], _i32),
        "sky_build_grid": ([_vp, _i64, _i32, _i64, P(Options), _vp, P(_vp)], _i32),
        "sky_prune_cells": ([_vp, _vp, _i32, _vp], _i32),
        "sky_grid_stats": ([_vp, P(GridStats)], _i32),
        "sky_grid_copy_out": ([_vp, _i32, _vp, _sz], _i32),
        "sky_grid_destroy": ([_vp], None),
        "sky_last_run_stats": ([P(RunStats)], _i32),
        "sky_set_phase_timing": ([_i32], _i32),
        "sky_last_phase_times": ([P(PhaseTimes)], _i32),
        "sky_status_string": ([_i32], ctypes.c_char_p),
        "sky_last_error": ([], ctypes.c_char_p),
        "sky_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != SKY_OK:
        raise SkyError(status, load().sky_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _opts(log2_g, assume_unit, filter_points, tile_cfg):
    o = Options()
    o.log2_g = -1 if log2_g is None else int(log2_g)
    # True -> 1 (Eq. 1 on the unit cube); False/0 -> automatic; 2 -> min/max normalisation
    o.assume_unit = int(assume_unit) if not isinstance(assume_unit, bool) else (1 if assume_unit else 0)
    o.tile_cfg = int(tile_cfg)
    if filter_points is not None and filter_points.numel() > 0:
        assert filter_points.is_cuda and filter_points.dtype == _torch().float32
        assert filter_points.is_contiguous()
        o.d_filter_pts = filter_points.data_ptr()
        o.n_filter = int(filter_points.shape[0])
    return o


def _points(points, dev=True):
    torch = _torch()
    if points.dim() == 1:
        points = points.view(-1, 1)
    if points.dim() != 2 or points.dtype != torch.float32:
        raise ValueError("points must be a 2-D float32 tensor")
    if dev and not points.is_cuda:
        raise ValueError("points must live on a CUDA device")
    if points.stride(1) != 1:
        raise ValueError("points must have unit column stride")
    n, d = points.shape
    ld = points.stride(0) if n > 1 else d
    return points, n, d, ld


def skyline(points, log2_g=None, assume_unit=False, filter_points=None, capacity=None,
            tile_cfg=0, stream=None, out=None):
    """Steps (a)-(d) on device-resident points: ascending int32 row ids (cuda)."""
    torch = _torch()
    lib = load()
    points, n, d, ld = _points(points)
    cap = n if capacity is None else int(capacity)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int32, device=points.device)
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, filter_points, tile_cfg)
    with torch.cuda.device(points.device):
        st = lib.sky_skyline(_vp(points.data_ptr()), n, d, ld, ctypes.byref(o), _vp(out.data_ptr()), cap,
                             ctypes.byref(cnt), _stream_ptr(stream))
    if st == 3:
        raise SkyError(st, f"{lib.sky_last_error().decode()} (count={cnt.value})")
    _check(st)
    return out[:cnt.value]


def skyline_host(points, log2_g=None, assume_unit=False, capacity=None, tile_cfg=0, stream=None, out=None):
    """Same result from host (ideally pinned) memory: copies in, computes, copies out.
    `points` is a CPU float32 torch tensor; returns a CPU int32 tensor."""
    torch = _torch()
    lib = load()
    points, n, d, ld = _points(points, dev=False)
    cap = n if capacity is None else int(capacity)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int32, pin_memory=points.is_pinned())
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, None, tile_cfg)
    st = lib.sky_skyline_host(_vp(points.data_ptr()), n, d, ld, ctypes.byref(o), _vp(out.data_ptr()), cap,
                              ctypes.byref(cnt), _stream_ptr(stream))
    _check(st)
    return out[:cnt.value]


def last_run_stats() -> dict:
    s = RunStats()
    _check(load().sky_last_run_stats(ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in RunStats._fields_}


def set_phase_timing(enable: bool = True):
    """Record CUDA events between the phases of later skyline calls on this thread."""
    _check(load().sky_set_phase_timing(1 if enable else 0))


def last_phase_times() -> dict:
    t = PhaseTimes()
    _check(load().sky_last_phase_times(ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in PhaseTimes._fields_}


class Grid:
    """Steps (a)-(c) with inspectable intermediate arrays (sky_build_grid & co)."""

    def __init__(self, points, log2_g=None, assume_unit=False, stream=None):
        torch = _torch()
        self._lib = load()
        self.points, self.n, self.d, self.ld = _points(points)
        self._stream = stream
        self._h = _vp()
        o = _opts(log2_g, assume_unit, None, 0)
        with torch.cuda.device(points.device):
            _check(self._lib.sky_build_grid(_vp(self.points.data_ptr()), self.n, self.d, self.ld,
                                            ctypes.byref(o), _stream_ptr(stream), ctypes.byref(self._h)))

    def prune(self, filter_points=None):
        nf, ptr = 0, None
        if filter_points is not None and filter_points.numel() > 0:
            nf, ptr = int(filter_points.shape[0]), filter_points.data_ptr()
        _check(self._lib.sky_prune_cells(self._h, _vp(ptr), nf, _stream_ptr(self._stream)))
        return self

    def stats(self) -> dict:
        s = GridStats()
        _check(self._lib.sky_grid_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in GridStats._fields_}

    def _copy(self, which, count, dtype):
        torch = _torch()
        t = torch.empty(max(count, 1), dtype=dtype, device=self.points.device)
        _check(self._lib.sky_grid_copy_out(self._h, which, _vp(t.data_ptr()), t.numel() * t.element_size()))
        return t[:count]

    @property
    def words(self):
        return max(1, (1 << (self.stats()["log2_g"] * self.d)) // 32)

    def cell_keys(self):
        return self._copy(GRID_CELL_KEY, self.n, _torch().int32)

    def occupied(self):
        return self._copy(GRID_OCCUPIED, self.words, _torch().int32)

    def dominated(self):
        return self._copy(GRID_DOMINATED, self.words, _torch().int32)

    def survivors(self):
        return self._copy(GRID_SURVIVORS, int(self.stats()["surviving_points"]), _torch().int32)

    def cell_map(self):
        return self._copy(GRID_CELL_MAP, 32, _torch().float32)

    def close(self):
        if self._h:
            self._lib.sky_grid_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().sky_version().decode()
