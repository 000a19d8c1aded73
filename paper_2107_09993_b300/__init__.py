"""Python binding of libsky (include/sky.h): exact SkyCell skyline on one GPU.

This module only marshals arguments: torch tensors in, torch tensors out.
Every step of the skyline path runs in the CUDA kernels of libsky.so
(compiled for sm_103a by ``build.py``). There is no CPU fallback: if the
library or a CUDA device is missing, every call raises.

    import paper_2107_09993_b300 as sky
    idx = sky.skyline(points_cuda_f32)          # ascending int32 row ids

Names follow the C ABI: ``skyline`` (sky_skyline), ``skyline_host``
(sky_skyline_host), ``skyline_witness`` (sky_skyline_witness), ``skyline_sets`` / ``skyline_host_sets``
(sky_skyline_sets / sky_skyline_host_sets), ``Grid`` (sky_build_grid / sky_prune_cells /
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
GRID_CELL_KEY, GRID_OCCUPIED, GRID_DOMINATED, GRID_SURVIVORS, GRID_CELL_MAP, GRID_SNAP = range(6)

_i32, _i64, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t


class SkyError(RuntimeError):
    def __init__(self, status: int, detail: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {detail}")


class Options(ctypes.Structure):
    _fields_ = [("log2_g", _i32), ("assume_unit", _i32), ("d_filter_pts", _vp),
                ("n_filter", _i32), ("survivors_only", _i32)]


class GridStats(ctypes.Structure):
    _fields_ = [("log2_g", _i32), ("d", _i32), ("n", _i64), ("occupied_cells", _i64),
                ("surviving_cells", _i64), ("surviving_points", _i64), ("n_filter_used", _i32),
                ("error_flags", _i32)]


class RunStats(ctypes.Structure):
    _fields_ = [("n", _i64), ("d", _i32), ("log2_g", _i32), ("survivors", _i64), ("skyline", _i64),
                ("pairs", _i64), ("n_filter_used", _i32), ("kernels", _i32), ("tiles", _i64),
                ("group_scans", _i64), ("code_hits", _i64), ("exact_tests", _i64)]


class PhaseTimes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("normalize_ms", "map_mark_ms", "prune_ms", "survivors_ms",
                                               "sort_ms", "gather_ms", "refine_ms", "emit_ms", "call_ms")]


class SkySet(ctypes.Structure):
    """struct sky_set: one point set of sky_skyline_sets / sky_skyline_host_sets."""
    _fields_ = [("pts", _vp), ("n", _i64), ("d", _i32), ("reserved0", _i32), ("ld", _i64),
                ("out_idx", _vp), ("capacity", _i64), ("count", _i64), ("status", _i32), ("reserved1", _i32)]


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
        "sky_skyline_witness": ([_vp, _i64, _i32, _i64, P(Options), _vp, _i64, P(_i64), _vp, _vp], _i32),
        "sky_skyline_sets": ([P(SkySet), _i32, P(Options), _vp], _i32),
        "sky_skyline_host_sets": ([P(SkySet), _i32, P(Options), _vp], _i32),
        "sky_skyline_chunked": ([_vp, _i32, _i64, _i32, _i64, P(Options), _i64, _i64, _vp, _i64, P(_i64), _vp],
                                _i32),
        "sky_build_grid": ([_vp, _i64, _i32, _i64, P(Options), _vp, P(_vp)], _i32),
        "sky_prune_cells": ([_vp, _vp, _i32, _vp], _i32),
        "sky_grid_stats": ([_vp, P(GridStats)], _i32),
        "sky_grid_copy_out": ([_vp, _i32, _vp, _sz], _i32),
        "sky_grid_destroy": ([_vp], None),
        "sky_last_run_stats": ([P(RunStats)], _i32),
        "sky_set_wait_limit": ([ctypes.c_uint32], _i32),
        "sky_tournament_workspace_size": ([_i32, _i32], _sz),
        "sky_tournament_cells": ([_vp, _i32, _i32, _vp, _vp, _sz, _vp], _i32),
        "sky_set_phase_timing": ([_i32], _i32),
        "sky_last_phase_times": ([P(PhaseTimes)], _i32),
        "sky_status_string": ([_i32], ctypes.c_char_p),
        "sky_last_error": ([], ctypes.c_char_p),
        "sky_version": ([], ctypes.c_char_p),
        "sky_baseline_sequential": ([_vp, _i64, _i32, _i64, _i32, _i32, _vp, _i64, P(_i64), P(_i64)], _i32),
        "sky_baseline_key_cells": ([_vp, _i64, _i32, _i64, _i32, _i32, _vp, _i64, P(_i64)], _i32),
        "sky_baseline_last_error": ([], ctypes.c_char_p),
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


def _opts(log2_g, assume_unit, filter_points, survivors_only=False):
    o = Options()
    o.log2_g = -1 if log2_g is None else int(log2_g)
    # True -> 1 (Eq. 1 on the unit cube); False/0 -> automatic; 2 -> min/max normalisation
    o.assume_unit = int(assume_unit) if not isinstance(assume_unit, bool) else (1 if assume_unit else 0)
    o.survivors_only = 1 if survivors_only else 0
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
    n, d = points.shape
    if n > 0 and d > 1 and points.stride(1) != 1:
        raise ValueError("points must have unit column stride")
    ld = points.stride(0) if n > 1 else d
    return points, n, d, ld


def skyline(points, log2_g=None, assume_unit=False, filter_points=None, capacity=None,
            survivors_only=False, stream=None, out=None):
    """Steps (a)-(d) on device-resident points: ascending int32 row ids (cuda).
    survivors_only=True stops after step (c) and returns the candidates."""
    torch = _torch()
    lib = load()
    points, n, d, ld = _points(points)
    cap = n if capacity is None else int(capacity)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int32, device=points.device)
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, filter_points, survivors_only)
    with torch.cuda.device(points.device):
        st = lib.sky_skyline(_vp(points.data_ptr()), n, d, ld, ctypes.byref(o), _vp(out.data_ptr()), cap,
                             ctypes.byref(cnt), _stream_ptr(stream))
    if st == 3:
        raise SkyError(st, f"{lib.sky_last_error().decode()} (count={cnt.value})")
    _check(st)
    return out[:cnt.value]


def skyline_witness(points, log2_g=None, assume_unit=False, filter_points=None, stream=None):
    """sky_skyline_witness: (skyline row ids, witnesses), both int32 CUDA
    tensors. witnesses[i] is -1 for a skyline row, else the row of a point
    that dominates row i (Definition 1); -2 marks a row step (c) dropped
    without a witness (an error of the path)."""
    torch = _torch()
    lib = load()
    points, n, d, ld = _points(points)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    wit = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, filter_points)
    with torch.cuda.device(points.device):
        st = lib.sky_skyline_witness(_vp(points.data_ptr()), n, d, ld, ctypes.byref(o), _vp(out.data_ptr()), n,
                                     ctypes.byref(cnt), _vp(wit.data_ptr()), _stream_ptr(stream))
    _check(st)
    return out[:cnt.value], wit[:n]


def skyline_host(points, log2_g=None, assume_unit=False, capacity=None, stream=None, out=None):
    """Same result from host (ideally pinned) memory: copies in, computes, copies out.
    `points` is a CPU float32 torch tensor; returns a CPU int32 tensor."""
    torch = _torch()
    lib = load()
    points, n, d, ld = _points(points, dev=False)
    cap = n if capacity is None else int(capacity)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int32, pin_memory=points.is_pinned())
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, None)
    st = lib.sky_skyline_host(_vp(points.data_ptr()), n, d, ld, ctypes.byref(o), _vp(out.data_ptr()), cap,
                              ctypes.byref(cnt), _stream_ptr(stream))
    _check(st)
    return out[:cnt.value]


def _run_sets(fn, sets_pts, outs, capacity, o, stream, dev):
    torch = _torch()
    arr = (SkySet * max(1, len(sets_pts)))()
    keep = []
    for i, pts in enumerate(sets_pts):
        pts, n, d, ld = _points(pts, dev=dev)
        cap = n if capacity is None else int(capacity)
        out = outs[i] if outs is not None else None
        if out is None:
            out = (torch.empty(max(cap, 1), dtype=torch.int32, device=pts.device) if dev else
                   torch.empty(max(cap, 1), dtype=torch.int32, pin_memory=pts.is_pinned()))
        assert out.dtype == torch.int32 and out.is_contiguous() and out.numel() >= cap
        arr[i].pts, arr[i].n, arr[i].d, arr[i].ld = pts.data_ptr(), n, d, ld
        arr[i].out_idx, arr[i].capacity = out.data_ptr(), cap
        keep.append((pts, out))
    st = fn(arr, len(sets_pts), ctypes.byref(o), stream)
    if st == 3:
        raise SkyError(st, load().sky_last_error().decode())
    _check(st)
    return [out[:arr[i].count] for i, (_, out) in enumerate(keep)]


def skyline_sets(sets, log2_g=None, assume_unit=False, capacity=None, survivors_only=False, stream=None,
                 outs=None):
    """sky_skyline_sets: the skylines of several device-resident point sets
    (a list of float32 [n_i, d_i] CUDA tensors), run concurrently. Returns a
    list of ascending int32 row-id tensors (cuda), one per set."""
    torch = _torch()
    lib = load()
    o = _opts(log2_g, assume_unit, None, survivors_only)
    if not sets:
        return []
    with torch.cuda.device(sets[0].device):
        return _run_sets(lib.sky_skyline_sets, sets, outs, capacity, o, _stream_ptr(stream), True)


def skyline_host_sets(sets, log2_g=None, assume_unit=False, capacity=None, survivors_only=False, stream=None,
                      outs=None):
    """sky_skyline_host_sets: the same from host (ideally pinned) CPU tensors;
    the copy of one set's points overlaps the kernels of the previous set.
    Returns a list of CPU int32 row-id tensors."""
    lib = load()
    o = _opts(log2_g, assume_unit, None, survivors_only)
    if not sets:
        return []
    return _run_sets(lib.sky_skyline_host_sets, sets, outs, capacity, o, _stream_ptr(stream), False)


def skyline_chunked(points, log2_g=None, assume_unit=False, survivors_only=False, chunk_rows=0,
                    max_candidates=0, capacity=None, stream=None):
    """sky_skyline_chunked: skyline of a set beyond one in-core call, processed
    in chunks against one occupancy bitmap. `points` is a float32 [n, d] CUDA
    tensor (device input) or CPU tensor / numpy array (host input, streamed;
    pin it for speed). Returns ascending int64 row ids (CUDA tensor)."""
    torch = _torch()
    lib = load()
    if not isinstance(points, torch.Tensor):
        import numpy as np
        points = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32))
    host = not points.is_cuda
    if points.dim() == 1:
        points = points.view(-1, 1)
    assert points.dtype == torch.float32 and points.stride(1) == 1
    n, d = int(points.shape[0]), int(points.shape[1])
    ld = int(points.stride(0)) if n > 1 else d
    dev = points.device if not host else torch.device("cuda", torch.cuda.current_device())
    cap = n if capacity is None else int(capacity)
    out = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    cnt = _i64(0)
    o = _opts(log2_g, assume_unit, None, survivors_only)
    st = lib.sky_skyline_chunked(_vp(points.data_ptr()), 1 if host else 0, n, d, ld, ctypes.byref(o),
                                 int(chunk_rows), int(max_candidates), _vp(out.data_ptr()), cap,
                                 ctypes.byref(cnt), _stream_ptr(stream))
    if st == 3:
        raise SkyError(st, f"{lib.sky_last_error().decode()} (count={cnt.value})")
    _check(st)
    return out[:cnt.value]


def last_run_stats() -> dict:
    s = RunStats()
    _check(load().sky_last_run_stats(ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in RunStats._fields_}


def tournament_cells(occupied, d: int, log2_g: int, stream=None):
    """sky_tournament_cells (Algorithm 3 on one layer): `occupied` is the
    layer's occupancy bitmap as an int32 CUDA tensor of 32-bit words; returns
    a uint8 CUDA tensor of 2^(log2_g d) class bytes (bit 0 dominated, bit 1
    key cell, bit 2 candidate cell)."""
    torch = _torch()
    lib = load()
    n = 1 << (int(log2_g) * int(d))
    ws_bytes = lib.sky_tournament_workspace_size(int(d), int(log2_g))
    if ws_bytes == 0:
        raise SkyError(6 if d >= 1 and log2_g >= 0 else 1, f"no tournament for d={d}, log2_g={log2_g}")
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=occupied.device)
    off = (-ws.data_ptr()) % 256
    cls = torch.empty(n, dtype=torch.uint8, device=occupied.device)
    with torch.cuda.device(occupied.device):
        _check(lib.sky_tournament_cells(_vp(occupied.data_ptr()), int(d), int(log2_g), _vp(cls.data_ptr()),
                                        _vp(ws.data_ptr() + off), ws_bytes, _stream_ptr(stream)))
    torch.cuda.synchronize(occupied.device)   # the workspace is released on return
    return cls


def set_wait_limit(polls: int):
    """sky_set_wait_limit: poll limit of the pipeline's bounded device waits
    (a test aid for the timeout path; 0 restores the default)."""
    _check(load().sky_set_wait_limit(int(polls)))


def set_phase_timing(enable=True):
    """Device timing of later skyline calls on this thread: True or 1 = events
    between the phases (kernels launched one by one), 2 = events around the
    whole kernel sequence (graph replay kept; last_phase_times()["call_ms"]),
    False or 0 = off."""
    mode = 1 if enable is True else (0 if enable is False else int(enable))
    _check(load().sky_set_phase_timing(mode))


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

    def snap_rows(self, n_prop):
        """Row of the data point each of the first n_prop proposals was
        snapped to (-1: none), after prune(filter_points); numpy int64."""
        v = self._copy(GRID_SNAP, 16, _torch().int64).cpu().numpy().view("u8")[:n_prop]
        return [int(x & 0xffffffff) if x != 0xffffffffffffffff else -1 for x in v]

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


# ---------------------------------------------------------------- batched --
QUERY_QUADRANT = 1


class Query(ctypes.Structure):
    _fields_ = [("row_begin", _i64), ("row_count", _i64), ("dim_mask", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("origin", ctypes.c_float * 16)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("h_log2g", _vp), ("refine_ctas_per_sm", _i32), ("class_ctas", _i32 * 4),
                ("class_stages", _i32 * 4), ("class_code", _i32 * 4), ("concurrent_classes", _i32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_queries", _i32), ("kernels", _i32), ("graph_launches_per_call", _i32), ("reserved", _i32),
                ("points", _i64), ("survivors", _i64), ("skyline", _i64), ("pairs", _i64)]


def _load_batched():
    lib = load()
    if getattr(lib, "_batched_bound", False):
        return lib
    P = ctypes.POINTER
    sig = {
        "sky_batch_create": ([_vp, _i64, _i32, _i64, _i64, _vp, _i32, P(BatchTuning), P(_vp), P(_sz)], _i32),
        "sky_batched_workspace_size": ([_i64, _i32, _i64, _i64, _vp, _i32, P(BatchTuning)], _sz),
        "sky_batch_bind": ([_vp, _vp, _sz, _vp, _i64, _vp, _vp, _vp], _i32),
        "sky_skyline_batched": ([_vp, _vp], _i32),
        "sky_batch_stats": ([_vp, _vp, P(BatchStats)], _i32),
        "sky_batch_destroy": ([_vp], None),
        "sky_batch_last_error": ([], ctypes.c_char_p),
        "sky_batched_device_workspace_size": ([_i32, _i32, _i64], _sz),
        "sky_skyline_batched_device": ([_vp, _i64, _i32, _i64, _i64, _vp, _i32, _i64, _vp, _sz, _vp, _i64, _vp, _vp,
                                        _vp], _i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    lib._batched_bound = True
    return lib


def _bcheck(status: int):
    if status != SKY_OK:
        raise SkyError(status, _load_batched().sky_batch_last_error().decode())


class Batch:
    """Many skylines over row ranges x attribute subsets of one device table,
    run as one CUDA-graph launch (sky_batch_create / bind / sky_skyline_batched).

    table: 2-D float32 CUDA tensor, row-major (stride (ld, 1)) or column-major
    (stride (1, ld)). queries: int array [n_queries, 3] of (row_begin,
    row_count, dim_mask). origins (optional): float array [n_queries, 16];
    a row with any non-NaN value makes that query a quadrant query with that
    origin (values in the order of its selected columns). Results: global
    ascending row ids per query."""

    def __init__(self, table, queries, log2g=None, refine_ctas_per_sm=0, capacity=None, stream=None,
                 origins=None, tuning="cache"):
        """tuning: "cache" (default) applies the autotuner's cached choices
        for this GPU (tune.py) when the cache has them and no explicit
        log2g / refine_ctas_per_sm is given; None uses the library defaults;
        a dict gives the knobs directly: class_ctas, class_stages, class_code
        (lists of 4), concurrent_classes, layer_offset (per-query list or
        array added to the automatic layer)."""
        import numpy as np
        torch = _torch()
        lib = _load_batched()
        if table.dim() != 2 or table.dtype != torch.float32 or not table.is_cuda:
            raise ValueError("table must be a 2-D float32 CUDA tensor")
        self.table = table
        q = np.asarray(queries, dtype=np.int64).reshape(-1, 3)
        self.nq = q.shape[0]
        arr = (Query * max(self.nq, 1))()
        org = None if origins is None else np.asarray(origins, dtype=np.float32).reshape(self.nq, 16)
        for i in range(self.nq):
            arr[i].row_begin, arr[i].row_count, arr[i].dim_mask = int(q[i, 0]), int(q[i, 1]), int(q[i, 2]) & 0xffffffff
            arr[i].flags = 0
            if org is not None and not np.all(np.isnan(org[i])):
                arr[i].flags = QUERY_QUADRANT
                for k in range(16):
                    arr[i].origin[k] = float(0.0 if np.isnan(org[i, k]) else org[i, k])
        self._queries = arr
        tune = BatchTuning()
        self._lg = None
        knobs = None
        if isinstance(tuning, dict):
            knobs = tuning
        elif tuning == "cache" and log2g is None and not refine_ctas_per_sm:
            from . import tune as _tune
            knobs = _tune.settings(q)
        if knobs:
            for c in range(4):
                tune.class_ctas[c] = int(knobs.get("class_ctas", [0] * 4)[c])
                tune.class_stages[c] = int(knobs.get("class_stages", [0] * 4)[c])
                tune.class_code[c] = int(knobs.get("class_code", [0] * 4)[c])
            tune.concurrent_classes = int(knobs.get("concurrent_classes", 0))
            if log2g is None and knobs.get("log2g") is not None:
                log2g = knobs["log2g"]
        self.tuning = knobs
        if log2g is not None:
            self._lg = np.ascontiguousarray(np.asarray(log2g, dtype=np.int32).reshape(-1))
            assert self._lg.size == self.nq
            tune.h_log2g = self._lg.ctypes.data
        tune.refine_ctas_per_sm = int(refine_ctas_per_sm)
        self._h = _vp()
        ws = _sz(0)
        n_rows, n_cols = table.shape
        _bcheck(lib.sky_batch_create(_vp(table.data_ptr()), n_rows, n_cols, table.stride(0), table.stride(1),
                                     ctypes.cast(arr, _vp), self.nq, ctypes.byref(tune), ctypes.byref(self._h),
                                     ctypes.byref(ws)))
        dev = table.device
        self.ws_bytes = ws.value
        self.ws = torch.empty(max(self.ws_bytes, 1) + 256, dtype=torch.uint8, device=dev)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        total_rows = int(q[:, 1].sum()) if self.nq else 0
        self.capacity = total_rows if capacity is None else int(capacity)
        self.out = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.offsets = torch.zeros(self.nq + 1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(max(self.nq, 1), dtype=torch.int32, device=dev)
        with torch.cuda.device(dev):
            _bcheck(lib.sky_batch_bind(self._h, _vp(self._ws_ptr), self.ws_bytes, _vp(self.out.data_ptr()),
                                       self.capacity, _vp(self.offsets.data_ptr()), _vp(self.status.data_ptr()),
                                       _stream_ptr(stream)))

    def run(self, stream=None):
        """One CUDA-graph launch of the whole batch (asynchronous)."""
        _bcheck(_load_batched().sky_skyline_batched(self._h, _stream_ptr(stream)))

    def results(self):
        """Per-query ascending global row ids (CPU int32 arrays); synchronises."""
        torch = _torch()
        torch.cuda.synchronize(self.table.device)
        off = self.offsets.cpu().numpy()
        out = self.out.cpu().numpy()
        return [out[off[i]:off[i + 1]] for i in range(self.nq)]

    def query_status(self):
        return self.status[:self.nq].cpu().numpy()

    def stats(self, stream=None) -> dict:
        s = BatchStats()
        _bcheck(_load_batched().sky_batch_stats(self._h, _stream_ptr(stream), ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in BatchStats._fields_ if f != "reserved"}

    def close(self):
        if self._h:
            _load_batched().sky_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


QUERY_RECORD_BYTES = 88   # sizeof(sky_query): int64 row_begin, int64 row_count, uint32 dim_mask, uint32 flags,
                          # float origin[16]


def query_records(row_begin, row_count, dim_mask, origins=None):
    """sky_query records built on the device from CUDA tensors (row_begin,
    row_count: int64 [nq]; dim_mask: int [nq], the low 32 bits; origins:
    optional float32 [nq, 16], a row with any non-NaN value marks a quadrant
    query). Returns a uint8 CUDA tensor [nq, 88] without a host round trip."""
    torch = _torch()
    nq = row_begin.numel()
    dev = row_begin.device
    rec = torch.zeros(nq, QUERY_RECORD_BYTES // 4, dtype=torch.int32, device=dev)
    w64 = rec.view(torch.int64)
    w64[:, 0] = row_begin.to(torch.int64)
    w64[:, 1] = row_count.to(torch.int64)
    m = dim_mask.to(torch.int64) & 0xffffffff
    rec[:, 4] = torch.where(m >= 2 ** 31, m - 2 ** 32, m).to(torch.int32)
    if origins is not None:
        o = origins.to(device=dev, dtype=torch.float32).reshape(nq, 16)
        quad = ~torch.isnan(o).all(dim=1)
        rec[:, 5] = quad.to(torch.int32) * QUERY_QUADRANT
        rec[:, 6:22] = torch.nan_to_num(o, nan=0.0).view(torch.int32)
    return rec.view(torch.uint8)


class DeviceBatch:
    """Batched skylines planned on the device (sky_skyline_batched_device):
    the query records live in device memory, the workspace is sized from the
    bounds (n_queries, max_total_rows), and run() enqueues the whole batch
    without synchronising, so it can be recorded in a CUDA graph and the
    records rewritten on the device between launches."""

    def __init__(self, table, n_queries: int, max_total_rows: int, capacity=None):
        torch = _torch()
        lib = _load_batched()
        if table.dim() != 2 or table.dtype != torch.float32 or not table.is_cuda:
            raise ValueError("table must be a 2-D float32 CUDA tensor")
        self.table = table
        self.nq = int(n_queries)
        self.max_total_rows = int(max_total_rows)
        n_cols = table.shape[1]
        self.ws_bytes = lib.sky_batched_device_workspace_size(n_cols, self.nq, self.max_total_rows)
        if self.ws_bytes == 0:
            raise SkyError(1, "bad bounds for a device-planned batch")
        dev = table.device
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        self._ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.capacity = self.max_total_rows if capacity is None else int(capacity)
        self.out = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.offsets = torch.zeros(self.nq + 1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(max(self.nq, 1), dtype=torch.int32, device=dev)

    def run(self, records, stream=None):
        """Enqueues the batch for `records` (uint8 CUDA tensor [n_queries, 88],
        see query_records) on `stream` (asynchronous; no host copy)."""
        torch = _torch()
        if records.dtype != torch.uint8 or not records.is_cuda or records.numel() != self.nq * QUERY_RECORD_BYTES:
            raise ValueError("records must be a uint8 CUDA tensor of n_queries x 88 bytes")
        if not records.is_contiguous() or records.data_ptr() % 8:
            raise ValueError("records must be contiguous and 8-byte aligned")
        t = self.table
        with torch.cuda.device(t.device):
            _bcheck(_load_batched().sky_skyline_batched_device(
                _vp(t.data_ptr()), t.shape[0], t.shape[1], t.stride(0), t.stride(1), _vp(records.data_ptr()),
                self.nq, self.max_total_rows, _vp(self._ws_ptr), self.ws_bytes, _vp(self.out.data_ptr()),
                self.capacity, _vp(self.offsets.data_ptr()), _vp(self.status.data_ptr()), _stream_ptr(stream)))

    def results(self):
        """Per-query ascending global row ids (CPU int32 arrays); synchronises."""
        torch = _torch()
        torch.cuda.synchronize(self.table.device)
        off = self.offsets.cpu().numpy()
        out = self.out.cpu().numpy()
        return [out[off[i]:off[i + 1]] for i in range(self.nq)]

    def query_status(self):
        return self.status[:self.nq].cpu().numpy()


# ---------------------------------------------------------- learned proposal --
MLP_FEATURES, MLP_OUTPUTS, MLP_PARAMS = 636, 264, 62088


def _load_mlp():
    lib = load()
    if getattr(lib, "_mlp_bound", False):
        return lib
    sig = {
        "sky_features": ([_vp, _i64, _i32, _i64, _vp, _vp, _vp, _vp], _i32),
        "sky_features_work_floats": ([], _sz),
        "sky_mlp_work_floats": ([_i32], _sz),
        "sky_mlp_forward": ([_vp, _vp, _i32, _vp, _vp, _vp], _i32),
        "sky_mlp_backward": ([_vp, _vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp, _vp, _vp], _i32),
        "sky_mlp_adamw": ([_vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float, _vp], _i32),
        "sky_mlp_round": ([_vp, _vp, _i64, _vp], _i32),
        "sky_propose": ([_vp, _i64, _i32, _i64, _vp, ctypes.c_float, _i64, _vp, ctypes.POINTER(_i32), _vp, _vp],
                        _i32),
        "sky_propose_work_floats": ([], _sz),
        "sky_mlp_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    lib._mlp_bound = True
    return lib


def _mcheck(status: int):
    if status != SKY_OK:
        raise SkyError(status, _load_mlp().sky_mlp_last_error().decode())


def _p(t):
    return _vp(t.data_ptr())


def features(points, stream=None):
    """sky_features: (features[636], range[32]) float32 CUDA tensors."""
    torch = _torch()
    lib = _load_mlp()
    points, n, d, ld = _points(points)
    feat = torch.empty(MLP_FEATURES, dtype=torch.float32, device=points.device)
    rng = torch.empty(32, dtype=torch.float32, device=points.device)
    work = torch.empty(int(lib.sky_features_work_floats()), dtype=torch.float32, device=points.device)
    _mcheck(lib.sky_features(_p(points), n, d, ld, _p(feat), _p(rng), _p(work), _stream_ptr(stream)))
    return feat, rng


def mlp_forward(params_bf16, feat, stream=None):
    """sky_mlp_forward: outputs [B, 264] for features [B, 636] (params: uint16/bf16 CUDA tensor)."""
    torch = _torch()
    lib = _load_mlp()
    feat = feat.reshape(-1, MLP_FEATURES).contiguous()
    B = feat.shape[0]
    out = torch.empty((B, MLP_OUTPUTS), dtype=torch.float32, device=feat.device)
    work = torch.empty(int(lib.sky_mlp_work_floats(B)), dtype=torch.float32, device=feat.device)
    _mcheck(lib.sky_mlp_forward(_p(params_bf16), _p(feat), B, _p(out), _p(work), _stream_ptr(stream)))
    return out


def mlp_backward(params_bf16, feat, dims, labels, targets, masks, lam, stream=None):
    """sky_mlp_backward: (mean loss tensor[1], gradient[62088])."""
    torch = _torch()
    lib = _load_mlp()
    B = feat.shape[0]
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feat.device)
    loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
    work = torch.empty(int(lib.sky_mlp_work_floats(B)), dtype=torch.float32, device=feat.device)
    _mcheck(lib.sky_mlp_backward(_p(params_bf16), _p(feat.contiguous()), _p(dims), _p(labels), _p(targets),
                                 _p(masks), B, float(lam), _p(grad), _p(work), _p(loss), _stream_ptr(stream)))
    return loss, grad


def mlp_adamw(master, params_bf16, m, v, grad, step, lr, wd, stream=None):
    _mcheck(_load_mlp().sky_mlp_adamw(_p(master), _p(params_bf16), _p(m), _p(v), _p(grad), int(step), float(lr),
                                      float(wd), _stream_ptr(stream)))


def mlp_round(master, params_bf16, stream=None):
    _mcheck(_load_mlp().sky_mlp_round(_p(master), _p(params_bf16), master.numel(), _stream_ptr(stream)))


def propose(points, params_bf16, inflate=0.02, n_ref=0, stream=None):
    """sky_propose: (log2_g, proposals[16, d] CUDA tensor). n_ref: the set
    size the weights were trained at (0: use the network's layer as is)."""
    torch = _torch()
    lib = _load_mlp()
    points, n, d, ld = _points(points)
    prop = torch.empty((16, d), dtype=torch.float32, device=points.device)
    work = torch.empty(int(lib.sky_propose_work_floats()), dtype=torch.float32, device=points.device)
    lg = _i32(0)
    _mcheck(lib.sky_propose(_p(points), n, d, ld, _p(params_bf16), float(inflate), int(n_ref), _p(prop),
                            ctypes.byref(lg), _p(work), _stream_ptr(stream)))
    return int(lg.value), prop


# Rows per training set of the shipped weights (learned_weights.npz).
TRAIN_ROWS = 100_000


def skyline_learned(points, params_bf16, inflate=0.02, n_ref=TRAIN_ROWS, stream=None, out=None):
    """The learned path: sky_propose, then sky_skyline with the proposed layer
    and filter points. Same result as skyline(points), by construction."""
    lg, prop = propose(points, params_bf16, inflate, n_ref=n_ref, stream=stream)
    d = points.shape[1] if points.dim() == 2 else 1
    lg = max(1, min(lg, 27 // d, 16))
    return skyline(points, log2_g=lg, filter_points=prop, stream=stream, out=out)


# ------------------------------------------------------------ CPU baseline --
def _baseline_points(points):
    import numpy as np
    P = np.ascontiguousarray(points, dtype=np.float32)
    if P.ndim != 2:
        raise ValueError("points must be an n x d array")
    return P


def _baseline_check(status: int):
    if status != SKY_OK:
        raise SkyError(status, load().sky_baseline_last_error().decode())


def baseline_sequential(points, log2_g=None, assume_unit=False):
    """The paper's sequential SkyCell on the host (sky_baseline_sequential):
    a CPU comparison for the GPU path, not part of it. numpy n x d float32 in,
    (ascending int32 skyline row ids, candidates refined after the cell
    pruning) out."""
    import numpy as np
    lib = load()
    P = _baseline_points(points)
    n, d = P.shape
    out = np.empty(max(n, 1), dtype=np.int32)
    cnt, cand = _i64(0), _i64(0)
    st = lib.sky_baseline_sequential(_vp(P.ctypes.data), n, d, d, -1 if log2_g is None else int(log2_g),
                                     1 if assume_unit else 0, _vp(out.ctypes.data), out.size, ctypes.byref(cnt),
                                     ctypes.byref(cand))
    _baseline_check(st)
    return out[:cnt.value].copy(), int(cand.value)


def baseline_key_cells(points, log2_g, assume_unit=False):
    """Key cells (Def. 4) of Layer log2_g found by the sequential baseline's
    slice enumeration: ascending int64 cell keys."""
    import numpy as np
    lib = load()
    P = _baseline_points(points)
    n, d = P.shape
    cap = max(n, 1)
    out = np.empty(cap, dtype=np.int64)
    cnt = _i64(0)
    st = lib.sky_baseline_key_cells(_vp(P.ctypes.data), n, d, d, int(log2_g), 1 if assume_unit else 0,
                                    _vp(out.ctypes.data), cap, ctypes.byref(cnt))
    _baseline_check(st)
    return out[:cnt.value].copy()
