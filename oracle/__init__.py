"""CPU oracle for the SkyCell skyline path -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. It shares no code with the CUDA library and never
imports it; both sides take their inputs from ``skydata``.

The C part (``sky_oracle.c``) is built with gcc into ``liboracle.so`` next to
this file. The Python part marshals numpy arrays and adds the few pieces whose
plain definition is clearest in numpy (batched queries, the learned proposal's
features and network, see ``mlp.py``).

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against values the paper prints (Table 1, the Eq. 1 example, Fig. 1/2
reconstructions, Corollary 1 counts) and against invariants fixed by the
mathematics (d = 1, anti-chains, duplicates, brute force == SFS, metamorphic
transforms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sky_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_int = ctypes.c_int
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile sky_oracle.c with gcc (IEEE binary32, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fexcess-precision=standard", "-std=c11", "-Wall", "-shared", "-fPIC",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_dominates.argtypes = [_vp, _vp, _int]
        lib.orc_dominates.restype = _int
        for name in ("orc_skyline_brute", "orc_skyline_sfs"):
            f = getattr(lib, name)
            f.argtypes = [_vp, _i64, _int, _i64, _vp, _int]
            f.restype = _i64
        lib.orc_dominator.argtypes = [_vp, _i64, _int, _i64, _i64]
        lib.orc_dominator.restype = _i64
        lib.orc_dominators.argtypes = [_vp, _i64, _int, _i64, _vp, _i64, _vp, _int]
        lib.orc_dominators.restype = None
        lib.orc_cell_params.argtypes = [_vp, _i64, _int, _i64, _int, _int, _vp, _vp]
        lib.orc_cell_params.restype = None
        lib.orc_cell_keys.argtypes = [_vp, _i64, _int, _i64, _int, _vp, _vp, _vp]
        lib.orc_cell_keys.restype = None
        lib.orc_cell_classes.argtypes = [_vp, _int, _int, _vp, _vp, _vp]
        lib.orc_cell_classes.restype = _i64
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = _int
        _lib = lib
    return _lib


def _pts(P):
    P = np.asarray(P)
    if P.dtype != np.float32:
        P = P.astype(np.float32)
    if P.ndim == 1:
        P = P.reshape(-1, 1)
    P = np.ascontiguousarray(P)
    return P, P.shape[0], P.shape[1]


def max_threads() -> int:
    return int(_load().orc_max_threads())


def dominates(p, q) -> bool:
    """Definition 1."""
    p = np.ascontiguousarray(p, dtype=np.float32).ravel()
    q = np.ascontiguousarray(q, dtype=np.float32).ravel()
    assert p.size == q.size
    return bool(_load().orc_dominates(p.ctypes.data, q.ctypes.data, p.size))


def skyline_brute(P, threads: int = 0) -> np.ndarray:
    """Definition 2, literal O(n^2 d): ascending int32 indices of the skyline."""
    P, n, d = _pts(P)
    out = np.empty(max(n, 1), dtype=np.int32)
    s = _load().orc_skyline_brute(P.ctypes.data, n, d, d, out.ctypes.data, threads)
    if s < 0:
        raise MemoryError("oracle allocation failed")
    return out[:s].copy()


def skyline_sfs(P, threads: int = 0) -> np.ndarray:
    """Sort-first skyline (Sec. 2.1): same set as skyline_brute, faster."""
    P, n, d = _pts(P)
    out = np.empty(max(n, 1), dtype=np.int32)
    s = _load().orc_skyline_sfs(P.ctypes.data, n, d, d, out.ctypes.data, threads)
    if s < 0:
        raise MemoryError("oracle allocation failed")
    return out[:s].copy()


def dominator(P, i: int) -> int:
    """First j whose point dominates point i, or -1 (i is a skyline point)."""
    P, n, d = _pts(P)
    return int(_load().orc_dominator(P.ctypes.data, n, d, d, int(i)))


def dominators(P, idx, threads: int = 0) -> np.ndarray:
    """Vectorised `dominator` over an index sample (threads over the sample)."""
    P, n, d = _pts(P)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    w = np.empty(idx.size, dtype=np.int64)
    _load().orc_dominators(P.ctypes.data, n, d, d, idx.ctypes.data, idx.size,
                           w.ctypes.data, threads)
    return w


MAP_MODES = {"auto": 0, "unit": 1, "minmax": 2}


def _mode(assume_unit, mode):
    if mode is None:
        mode = "unit" if assume_unit else "minmax"
    return MAP_MODES[mode]


def cell_params(P, log2g: int, assume_unit: bool = False, mode: str | None = None):
    """Offsets and scales of the value->column map (float32 arrays of length d).
    mode: "unit" (Eq. 1 as printed), "minmax" (per-dimension normalisation
    over all rows) or "auto" (decided on the rows 0, t, 2t, ... with
    t = ceil(n / 4096): Eq. 1 when every sampled dimension lies in [0,1] and
    spans >= 0.5, else normalisation by the sample's min / max)."""
    P, n, d = _pts(P)
    off = np.empty(d, dtype=np.float32)
    sc = np.empty(d, dtype=np.float32)
    _load().orc_cell_params(P.ctypes.data, n, d, d, int(log2g), _mode(assume_unit, mode),
                            off.ctypes.data, sc.ctypes.data)
    return off, sc


def cell_keys(P, log2g: int, assume_unit: bool = False, mode: str | None = None) -> np.ndarray:
    """Eq. 1: uint64 key of each point's Layer-log2g cell (dim d-1 most significant)."""
    P, n, d = _pts(P)
    off, sc = cell_params(P, log2g, assume_unit, mode)
    keys = np.empty(n, dtype=np.uint64)
    _load().orc_cell_keys(P.ctypes.data, n, d, d, int(log2g), off.ctypes.data,
                          sc.ctypes.data, keys.ctypes.data)
    return keys


def cell_columns(key: int, d: int, log2g: int) -> tuple:
    """Column numbers (c[0], ..., c[d-1]) of a cell key."""
    m = (1 << log2g) - 1
    return tuple((int(key) >> (log2g * k)) & m for k in range(d))


def cell_key(cols, log2g: int) -> int:
    """Inverse of cell_columns: cols = (c[0], ..., c[d-1])."""
    key = 0
    for k in reversed(range(len(cols))):
        key = (key << log2g) | int(cols[k])
    return key


def occupancy(keys, d: int, log2g: int) -> np.ndarray:
    """occ[c] = 1 when some point falls in cell c (uint8 array of G^d)."""
    occ = np.zeros(1 << (log2g * d), dtype=np.uint8)
    occ[np.asarray(keys, dtype=np.int64)] = 1
    return occ


def dominated_cells(occ, d: int, log2g: int) -> np.ndarray:
    """Definition 3 through the box identity: cell c is dominated iff some
    occupied cell c' has c'[k] < c[k] in every dimension, i.e. iff the closed
    box [0, c - (1, ..., 1)] holds an occupied cell. The box indicator is the
    cumulative OR of the occupancy along every axis (numpy). uint8 array."""
    G = 1 << log2g
    occ = np.asarray(occ, dtype=bool)
    assert occ.size == G ** d
    box = occ.reshape((G,) * d)              # axis 0 is dimension d-1 (most significant)
    for ax in range(d):
        box = np.logical_or.accumulate(box, axis=ax)
    dom = np.zeros((G,) * d, dtype=np.uint8)
    dom[(slice(1, None),) * d] = box[(slice(0, -1),) * d]
    return dom.reshape(-1)


def cell_classes(occ, d: int, log2g: int):
    """Definitions 3-6 over one layer: (dominated, key, candidate, n_candidates)."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    ncell = 1 << (log2g * d)
    assert occ.size == ncell
    dom = np.zeros(ncell, dtype=np.uint8)
    key = np.zeros(ncell, dtype=np.uint8)
    cand = np.zeros(ncell, dtype=np.uint8)
    cnt = _load().orc_cell_classes(occ.ctypes.data, d, log2g, dom.ctypes.data,
                                   key.ctypes.data, cand.ctypes.data)
    return dom, key, cand, int(cnt)


def skyline_subset(table, row_begin: int, row_count: int, dim_mask: int,
                   threads: int = 0, method: str = "sfs", origin=None) -> np.ndarray:
    """Skyline of rows [row_begin, row_begin+row_count) over the columns in
    dim_mask, returned as ascending global row ids (int32).

    origin (quadrant query, the paper's query experiments in Sec. 7): the
    query point becomes the origin and only the rows in its upper quadrant
    (row >= origin in every selected column) take part; since Definition 1
    compares coordinates pairwise, shifting those rows by the origin leaves
    their skyline unchanged, so it is the skyline of the kept rows as they
    are."""
    cols = [k for k in range(table.shape[1]) if (dim_mask >> k) & 1]
    sub = np.ascontiguousarray(table[row_begin:row_begin + row_count][:, cols])
    keep = np.arange(sub.shape[0])
    if origin is not None:
        o = np.asarray(origin, dtype=np.float32)[:len(cols)]
        keep = np.flatnonzero(np.all(sub >= o, axis=1))
        sub = np.ascontiguousarray(sub[keep])
    f = skyline_sfs if method == "sfs" else skyline_brute
    return (keep[f(sub, threads)] + row_begin).astype(np.int32)


def snap_rows(P, F) -> np.ndarray:
    """The learned pre-filter's snap (the reading that keeps it exact: a
    proposal may only prune through a real data point). Proposal f becomes
    the data point q with q <= f in every dimension whose coordinate sum is
    smallest, the sum taken in IEEE binary32 in dimension order (k = 0, 1,
    ...), ties to the lower row; -1 when no point is <= f. Returns one row
    per proposal (int64)."""
    P, n, d = _pts(P)
    F = np.asarray(F, dtype=np.float32).reshape(-1, d)
    s = np.zeros(n, dtype=np.float32)
    for k in range(d):
        s = np.add(s, P[:, k], dtype=np.float32)     # binary32, round to nearest
    out = np.full(F.shape[0], -1, dtype=np.int64)
    for j, f in enumerate(F):
        idx = np.flatnonzero(np.all(P <= f, axis=1))
        if idx.size:
            sj = s[idx]
            out[j] = idx[np.flatnonzero(sj == sj.min())[0]]
    return out
