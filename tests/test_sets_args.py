"""CPU checks of the multi-set entry points (sky_skyline_sets,
sky_skyline_host_sets): every set's arguments are checked before any device
work, and the failing set is named."""
import ctypes

import pytest


def _lib():
    import paper_2107_09993_b300 as sky
    return sky, sky.load()


def _arr(sky, specs):
    arr = (sky.SkySet * len(specs))()
    bufs = []
    for i, (n, d, ld, cap) in enumerate(specs):
        pts = (ctypes.c_float * max(1, n * ld))()
        out = (ctypes.c_int32 * max(1, cap))()
        bufs.append((pts, out))
        arr[i].pts = ctypes.addressof(pts)
        arr[i].n, arr[i].d, arr[i].ld = n, d, ld
        arr[i].out_idx, arr[i].capacity = ctypes.addressof(out), cap
        arr[i].count, arr[i].status = 123, 77
    return arr, bufs


@pytest.mark.parametrize("fn", ["sky_skyline_sets", "sky_skyline_host_sets"])
def test_bad_set_is_named_before_any_work(fn):
    sky, lib = _lib()
    arr, _keep = _arr(sky, [(10, 3, 3, 10), (10, 4, 4, 10), (10, 17, 17, 10)])
    st = getattr(lib, fn)(arr, 3, None, None)
    assert st == 1
    assert lib.sky_last_error().startswith(b"set 2: d = 17")
    # nothing ran: the outputs are untouched
    assert [(a.count, a.status) for a in arr] == [(123, 77)] * 3

    arr, _keep = _arr(sky, [(10, 3, 2, 10)])   # ld < d
    assert getattr(lib, fn)(arr, 1, None, None) == 1
    assert lib.sky_last_error().startswith(b"set 0: ld")

    arr, _keep = _arr(sky, [(10, 3, 3, 10)])
    arr[0].out_idx = None                      # capacity without a buffer
    assert getattr(lib, fn)(arr, 1, None, None) == 1
    assert b"set 0" in lib.sky_last_error()


@pytest.mark.parametrize("fn", ["sky_skyline_sets", "sky_skyline_host_sets"])
def test_options_checked_for_every_set(fn):
    sky, lib = _lib()
    arr, _keep = _arr(sky, [(10, 3, 3, 10), (10, 9, 9, 10)])
    o = sky.Options()
    o.log2_g = 3                               # 3 * 9 = 27 bits: fits
    o.assume_unit = 1
    o.log2_g = 4                               # 4 * 9 = 36 bits: too large for set 1
    st = getattr(lib, fn)(arr, 2, ctypes.byref(o), None)
    assert st == 6
    assert lib.sky_last_error().startswith(b"set 1:")
    o = sky.Options()
    o.n_filter = 2                             # proposals belong to one set
    o.d_filter_pts = 16
    assert getattr(lib, fn)(arr, 2, ctypes.byref(o), None) == 1
    assert b"n_filter" in lib.sky_last_error()


def test_empty_call_and_bad_count():
    sky, lib = _lib()
    assert lib.sky_skyline_sets(None, 0, None, None) == 0
    assert lib.sky_skyline_host_sets(None, 0, None, None) == 0
    assert lib.sky_skyline_sets(None, -1, None, None) == 1
    assert lib.sky_skyline_sets(None, 2, None, None) == 1
