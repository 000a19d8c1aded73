"""The timeout path of the bounded device waits (failure detection on the GPU
without a fault): with the pipeline's poll limit set to 1 by
sky_set_wait_limit, the waits of the streaming stages and look-back flags run
out; the kernels record the timeout, let their own bulk copies land (those
waits keep the default limit) and return; the call reports SKY_ERR_TIMEOUT.
Then, with the default limit restored, the next call on the same device and
the same buffers returns the oracle's skyline."""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402

TIMEOUT = 7   # SKY_ERR_TIMEOUT


def _expect_timeout(fn, tries=3):
    for _ in range(tries):
        try:
            fn()
        except sky.SkyError as e:
            assert e.status == TIMEOUT, e
            return True
    return False


def test_single_set_times_out_then_recovers():
    P = skydata.anticorrelated(200_000, 8, seed=4)
    x = torch.from_numpy(P).cuda()
    want = oracle.skyline_sfs(P)
    assert np.array_equal(sky.skyline(x).cpu().numpy(), want)
    assert np.array_equal(sky.skyline(x).cpu().numpy(), want)   # the cached graph from here on
    sky.set_wait_limit(1)
    try:
        assert _expect_timeout(lambda: sky.skyline(x))
    finally:
        sky.set_wait_limit(0)
    assert np.array_equal(sky.skyline(x).cpu().numpy(), want)
    torch.cuda.synchronize()


def test_sets_and_batched_report_timeouts_then_recover():
    P = [skydata.generate(k, 100_000, 6, 7) for k in ("independent", "anticorrelated")]
    xs = [torch.from_numpy(p).cuda() for p in P]
    want = [oracle.skyline_sfs(p) for p in P]
    T = skydata.mixed_table(200_000, 8, seed=3)
    q = skydata.batched_queries(64, T.shape[0], T.shape[1], seed=5, n_lo=1000, n_hi=100_000, d_lo=2, d_hi=8)
    b = sky.Batch(torch.from_numpy(T).cuda(), q)
    b.run()
    sky.set_wait_limit(1)
    try:
        assert _expect_timeout(lambda: sky.skyline_sets(xs))
        seen = False
        for _ in range(3):
            b.run()
            torch.cuda.synchronize()
            if np.any(b.query_status() == TIMEOUT):
                seen = True
                break
        assert seen
    finally:
        sky.set_wait_limit(0)
    got = [r.cpu().numpy() for r in sky.skyline_sets(xs)]
    assert all(np.array_equal(g, w) for g, w in zip(got, want))
    b.run()
    assert np.all(b.query_status() == 0)
    res = b.results()
    for i in (0, 17, 63):
        r0, c, m = (int(v) for v in q[i])
        assert res[i].tolist() == oracle.skyline_subset(T, r0, c, m).tolist()
    b.close()


def _stale_pool(nbytes=256 << 20):
    """Leaves nbytes of 0xFF bytes in CUDA's default memory pool, where the
    library's next workspaces come from (its pool keeps freed memory)."""
    from cuda.bindings import runtime as rt
    err, ptr = rt.cudaMallocAsync(nbytes, 0)
    assert err == rt.cudaError_t.cudaSuccess
    assert rt.cudaMemsetAsync(ptr, 0xFF, nbytes, 0)[0] == rt.cudaError_t.cudaSuccess
    assert rt.cudaFreeAsync(ptr, 0)[0] == rt.cudaError_t.cudaSuccess
    assert rt.cudaStreamSynchronize(0)[0] == rt.cudaError_t.cudaSuccess


def test_first_call_times_out_on_a_stale_workspace():
    """A call whose map pass gives up before writing every row's cell key,
    on a workspace of 0xFF bytes (rows it did not reach keep the key
    0xFFFFFFFF): the later kernels must stay inside their arrays (the cell
    keys are masked to the grid), the call reports SKY_ERR_TIMEOUT, and the
    next call with the default limit returns the oracle's skyline."""
    P = [skydata.generate(k, 150_000, 7, 9) for k in ("independent", "anticorrelated")]
    want = [oracle.skyline_sfs(p) for p in P]
    xs = [torch.from_numpy(p).cuda() for p in P]
    torch.cuda.synchronize()
    _stale_pool()
    sky.set_wait_limit(1)
    try:
        assert _expect_timeout(lambda: sky.skyline_sets(xs))
    finally:
        sky.set_wait_limit(0)
    got = [r.cpu().numpy() for r in sky.skyline_sets(xs)]
    assert all(np.array_equal(g, w) for g, w in zip(got, want))
