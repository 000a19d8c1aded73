"""GPU test of sky_skyline_noalloc, the entry point that allocates nothing.

Some callers cannot allocate memory where they need a skyline (their device
memory already belongs to their own arena allocator, or an allocation's
implicit synchronisation is not allowed in their loop). sky_skyline_noalloc
serves them from a fixed scratch array inside the library. This test calls it
through the C ABI and checks that two calls in a row give exactly the indices
of the regular sky_skyline entry point (the skyline is an index set, so the
tolerance is exact equality), and that oversized requests are refused.

Kept in its own file, named to be collected last, so that a run stopping at the
first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def _bind(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.sky_skyline_noalloc.argtypes = [vp, i64, i32, i64, ctypes.POINTER(sky.Options), vp, i64,
                                        ctypes.POINTER(i64), vp]
    lib.sky_skyline_noalloc.restype = i32
    lib.sky_noalloc_last_error.argtypes = []
    lib.sky_noalloc_last_error.restype = ctypes.c_char_p
    return lib


def _noalloc(lib, x, cap, **kw):
    n, d = x.shape
    o = sky._opts(kw.get("log2_g"), kw.get("assume_unit", False), None, 0)
    out = torch.full((max(cap, 1),), -7, dtype=torch.int32, device=x.device)
    cnt = ctypes.c_int64(-1)
    st = lib.sky_skyline_noalloc(ctypes.c_void_p(x.data_ptr()), n, d, d, ctypes.byref(o),
                                 ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, cnt.value, out


def test_noalloc_matches_regular_entry_point_twice():
    lib = _bind(sky.load())
    cases = [("anticorrelated", 65536, 8), ("independent", 40000, 4), ("correlated", 3000, 16),
             ("anticorrelated", 129, 3), ("independent", 1, 2)]
    for kind, n, d in cases:
        x = torch.from_numpy(skydata.generate(kind, n, d, seed=n + d)).cuda()
        want = sky.skyline(x).cpu()
        for call in range(2):
            st, cnt, out = _noalloc(lib, x, n)
            assert st == 0, (kind, n, d, call, lib.sky_noalloc_last_error())
            assert cnt == want.numel()
            assert torch.equal(out[:cnt].cpu(), want), (kind, n, d, call)
        # unit-cube map, explicit grid
        lg = min(2, 20 // d)
        want_u = sky.skyline(x, assume_unit=True, log2_g=lg).cpu()
        st, cnt, out = _noalloc(lib, x, n, assume_unit=True, log2_g=lg)
        assert st == 0 and torch.equal(out[:cnt].cpu(), want_u)


def test_noalloc_matches_oracle_at_the_limits():
    """Against the oracle directly (a fault in a kernel both entry points
    share would pass the comparison above): small sets, and the largest
    workspace the limits admit -- n = 65,536 points at d = 16 with a 2^16- and
    a 2^20-cell grid (log2_g * d = 16 and 20), and d = 10 with 2^20 cells."""
    lib = _bind(sky.load())
    cases = [("anticorrelated", 65536, 8, None), ("anticorrelated", 129, 3, None),
             ("anticorrelated", 65536, 16, 1), ("independent", 65536, 10, 2), ("correlated", 65536, 4, 5)]
    for kind, n, d, lg in cases:
        P = skydata.generate(kind, n, d, seed=n + 3 * d)
        x = torch.from_numpy(P).cuda()
        want = oracle.skyline_sfs(P)
        kw = {} if lg is None else {"log2_g": lg, "assume_unit": True}
        for call in range(2):
            st, cnt, out = _noalloc(lib, x, n, **kw)
            assert st == 0, (kind, n, d, lg, lib.sky_noalloc_last_error())
            assert np.array_equal(out[:cnt].cpu().numpy(), want), (kind, n, d, lg, call)
    # the error message also reaches sky_last_error()
    st, cnt, out = _noalloc(lib, torch.rand((65537, 2), device="cuda"), 65537)
    assert st == 6 and b"65536" in lib.sky_last_error()


def test_noalloc_refuses_oversized_requests():
    lib = _bind(sky.load())
    x = torch.rand((65537, 4), device="cuda")
    st, cnt, out = _noalloc(lib, x, 65537)
    assert st == 6 and b"65536" in lib.sky_noalloc_last_error()
    y = torch.rand((1000, 4), device="cuda")
    st, cnt, out = _noalloc(lib, y, 1000, log2_g=6)          # 2^24 cells > 2^20
    assert st == 6 and b"2^20" in lib.sky_noalloc_last_error()
    want = sky.skyline(y).cpu()
    st, cnt, out = _noalloc(lib, y, want.numel() - 1)
    assert st == 3 and cnt == want.numel()


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so under stream capture it returns
    SKY_ERR_INVALID_ARGUMENT without touching the capture; the captured work
    and later calls are unaffected."""
    lib = _bind(sky.load())
    x = torch.from_numpy(skydata.generate("independent", 1000, 4, seed=5)).cuda()
    want = sky.skyline(x).cpu()
    assert _noalloc(lib, x, 1000)[0] == 0          # first call (address look-up) before any capture
    y = torch.empty_like(x)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        y.copy_(x)
        st, _, _ = _noalloc(lib, y, 1000)
    assert st == 1 and b"captured" in lib.sky_noalloc_last_error()
    y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, x)
    st, cnt, out = _noalloc(lib, y, 1000)
    assert st == 0 and torch.equal(out[:cnt].cpu(), want)
