"""CPU checks of the workspace bound of the batch planned on the device
(sky_batched_device_workspace_size, a host function: no GPU needed).

The device planner lays out, per query, the arrays the batched kernels use
(result block, bitmap, look-back states, keep bytes, digit totals, layer-1
cell index of 2 * 2^d words, keys,
prefix-OR, four sort arrays, histograms, coordinates, codes, ids, sub-tile
minima, tile ends, super-tile minima, stage, and from 12 padded dimensions
the refinement's threshold masks of 16 bytes a padded row), each rounded up to 256 bytes,
after a header (plans, chunk and tile prefixes, work items, class table,
offsets, counters). It refuses a batch whose arrays do not fit. The bound must
therefore cover every batch whose valid queries hold at most max_total_rows
rows, whatever their sizes and dimensions; this file restates the layout
from those rules and checks the bound against it on random mixes."""
import math

import numpy as np
import pytest

A = 256
SCAN_TILE, REFINE_TILE = 2048, 128
PLAN_BYTES = 400          # sizeof(QueryPlan)
RESULT_BYTES = 72         # sizeof(DevResult)


def a256(x):
    return (x + A - 1) // A * A


def pad4(d):
    return (d + 3) // 4 * 4


def auto_layer(n, d):
    r = max(1, min(8, 24 // d))
    while r > 1 and (1 << (r * d)) > 32 * max(n, 1):
        r -= 1
    while r > 1 and r * d > 18:
        r -= 1
    return r


def query_bytes(n, d):
    dp = pad4(d)
    words = max(1, (1 << (auto_layer(n, d) * d)) // 32)
    nn = max(n, 1)
    ch = max(1, math.ceil(n / SCAN_TILE))
    tl = max(1, math.ceil(n / REFINE_TILE))
    npad = tl * REFINE_TILE
    sizes = [RESULT_BYTES, 4 * words, 8 * ch, 8 * ch, nn + 16, 4 * 256 * 4, 8 << d,
             8 * nn, 4 * words, 4 * nn, 4 * nn, 4 * nn, 4 * nn, 4 * 256 * ch,
             4 * npad * dp, npad * dp, 4 * npad, 4 * tl * 5 * (dp // 4) + 16, 4 * tl,
             4 * math.ceil(tl / 32) * (dp // 4), 4 * nn, 16 * npad if dp >= 12 else 0]
    return sum(a256(s) for s in sizes)


def header_bytes(nq, max_rows):
    max_items = max_rows // REFINE_TILE + nq + 1
    return (a256(PLAN_BYTES * nq) + 2 * a256(8 * (nq + 1)) + a256(8 * max_items) + a256(32)
            + 2 * a256(8 * nq) + a256(32))


@pytest.fixture(scope="module")
def ws_size():
    import ctypes
    from paper_2107_09993_b300 import build as b
    lib = ctypes.CDLL(b.build())
    f = lib.sky_batched_device_workspace_size
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    f.restype = ctypes.c_size_t
    return f


def test_bound_covers_random_batches(ws_size):
    rng = np.random.default_rng(11)
    for trial in range(300):
        n_cols = int(rng.integers(1, 33))
        nq = int(rng.integers(1, 600))
        # log-uniform sizes, some empty, some tiny, a few large
        n = np.exp(rng.uniform(0, np.log(2e6), nq)).astype(np.int64)
        n[rng.random(nq) < 0.05] = 0
        d = rng.integers(1, min(16, n_cols) + 1, nq)
        total = int(n.sum())
        need = header_bytes(nq, total) + sum(query_bytes(int(a), int(b)) for a, b in zip(n, d))
        assert ws_size(n_cols, nq, total) >= need, (trial, n_cols, nq, total)


def test_bound_at_the_extremes(ws_size):
    for n_cols in (1, 4, 12, 16, 32):
        dmax = min(16, n_cols)
        for nq, rows in ((1, 0), (1, 1), (1, 127), (1, 129), (1, 2049), (7, 10**7), (4096, 6 * 10**8)):
            sizes = [rows // nq] * nq
            sizes[0] += rows - sum(sizes)
            need = header_bytes(nq, rows) + sum(query_bytes(s, dmax) for s in sizes)
            assert ws_size(n_cols, nq, rows) >= need, (n_cols, nq, rows)
            # every query of the widest class, and one of one dimension
            need1 = header_bytes(nq, rows) + sum(query_bytes(s, 1) for s in sizes)
            assert ws_size(n_cols, nq, rows) >= need1


def test_bound_is_monotone_and_rejects_bad_arguments(ws_size):
    prev = 0
    for rows in (0, 10, 10**3, 10**5, 10**7):
        w = ws_size(12, 64, rows)
        assert w > prev
        prev = w
    assert ws_size(12, 128, 10**5) > ws_size(12, 64, 10**5)
    assert ws_size(16, 64, 10**5) >= ws_size(4, 64, 10**5)
    assert ws_size(0, 4, 100) == 0 and ws_size(33, 4, 100) == 0
    assert ws_size(8, -1, 100) == 0 and ws_size(8, 4, -1) == 0
    # the 4,096-query workload (6.05e8 rows, 12 columns) fits a B300 with room to spare
    assert ws_size(12, 4096, 605_000_000) < 100 * 2**30
