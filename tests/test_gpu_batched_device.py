"""The batch planned on the device (sky_skyline_batched_device): query records
in device memory, workspace from bounds, no host round trip. Every comparison
is exact equality of ascending global row-id arrays, against the host-planned
batch and the CPU oracle."""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def _records(q, origins=None):
    q = torch.as_tensor(np.asarray(q, dtype=np.int64).reshape(-1, 3)).cuda()
    o = None if origins is None else torch.as_tensor(np.asarray(origins, dtype=np.float32)).cuda()
    return sky.query_records(q[:, 0], q[:, 1], q[:, 2], o)


def _host(t, q, origins=None):
    b = sky.Batch(t, q, origins=origins, tuning=None)
    b.run()
    res, st = b.results(), b.query_status()
    b.close()
    return res, st


@pytest.mark.parametrize("layout", ["row", "col"])
def test_device_batch_matches_host_batch_and_oracle(layout):
    T = skydata.mixed_table(60000, 12, 5)
    q = skydata.batched_queries(300, T.shape[0], T.shape[1], seed=3, n_lo=1, n_hi=20000, d_lo=1, d_hi=12)
    q[0] = (0, 0, 0b101)                 # empty query
    q[1] = (17, 1, 0b1)                  # one row, one column
    q[2] = (0, T.shape[0], 0xfff)        # the whole table, all 12 columns
    q[3] = (T.shape[0] - 5, 5, 0b100000000001)
    t = torch.from_numpy(T).cuda()
    if layout == "col":
        t = t.t().contiguous().t()
    total = int(q[:, 1].sum())
    db = sky.DeviceBatch(t, len(q), total)
    db.run(_records(q))
    got, st = db.results(), db.query_status()
    want, wst = _host(t, q)
    assert st.tolist() == [0] * len(q) and wst.tolist() == [0] * len(q)
    for i in range(len(q)):
        assert np.array_equal(got[i], want[i]), i
    off = db.offsets.cpu().numpy()
    assert off[0] == 0 and off[-1] == sum(len(r) for r in got)
    for i in (0, 1, 2, 3, 50, 299):     # the oracle on a few queries
        b, c, m = (int(v) for v in q[i])
        assert got[i].tolist() == oracle.skyline_subset(T, b, c, m).tolist(), i


def test_device_batch_quadrant_queries():
    T = skydata.mixed_table(40000, 12, 6)
    q = skydata.batched_queries(64, T.shape[0], T.shape[1], seed=8, n_lo=100, n_hi=15000, d_lo=2, d_hi=8)
    rng = np.random.default_rng(4)
    org = np.full((len(q), 16), np.nan, dtype=np.float32)
    for i in range(0, len(q), 2):
        d = bin(int(q[i, 2])).count("1")
        org[i, :d] = rng.uniform(0.0, 0.4, d)
    t = torch.from_numpy(T).cuda()
    db = sky.DeviceBatch(t, len(q), int(q[:, 1].sum()))
    db.run(_records(q, org))
    got, st = db.results(), db.query_status()
    want, _ = _host(t, q, org)
    assert st.tolist() == [0] * len(q)
    for i in range(len(q)):
        assert np.array_equal(got[i], want[i]), i


def test_device_batch_invalid_queries_report_status():
    T = skydata.mixed_table(20000, 10, 7)
    q = skydata.batched_queries(40, T.shape[0], T.shape[1], seed=2, n_lo=10, n_hi=5000, d_lo=1, d_hi=10)
    bad = {3: (0, 10, 0), 7: (0, 10, 1 << 10), 11: (19990, 11, 0b11), 15: (-1, 5, 0b1),
           19: (0, 100, (1 << 17) - 1)}   # no column / missing column / rows past the end / negative / 17 dims
    for i, r in bad.items():
        q[i] = r
    t = torch.from_numpy(T).cuda()
    db = sky.DeviceBatch(t, len(q), 40 * 5000)
    db.run(_records(q))
    got, st = db.results(), db.query_status()
    good = [i for i in range(len(q)) if i not in bad]
    want, _ = _host(t, q[good])
    for i in bad:
        assert st[i] == 1 and got[i].size == 0, i
    for j, i in enumerate(good):
        assert st[i] == 0 and np.array_equal(got[i], want[j]), i


def test_device_batch_beyond_row_bound_runs_nothing():
    T = skydata.mixed_table(20000, 8, 9)
    q = np.array([(0, 12000, 0xff), (5000, 9000, 0b1011)], dtype=np.int64)
    t = torch.from_numpy(T).cuda()
    db = sky.DeviceBatch(t, 2, 20000)          # 21,000 rows asked for, bound 20,000
    db.run(_records(q))
    st = db.query_status()
    assert st.tolist() == [6, 6]
    assert db.offsets.cpu().tolist() == [0, 0, 0]
    # within the bound the same object runs them
    q[1, 1] = 8000
    db.run(_records(q))
    got, st = db.results(), db.query_status()
    assert st.tolist() == [0, 0]
    want, _ = _host(t, q)
    assert all(np.array_equal(a, b) for a, b in zip(got, want))


def test_device_batch_capacity_status():
    T = skydata.mixed_table(30000, 8, 10)
    q = np.array([(0, 30000, 0xff), (0, 30000, 0b11)], dtype=np.int64)
    t = torch.from_numpy(T).cuda()
    want, _ = _host(t, q)
    cap = len(want[0]) + len(want[1]) - 1
    db = sky.DeviceBatch(t, 2, 60000, capacity=cap)
    db.run(_records(q))
    st = db.query_status()
    off = db.offsets.cpu().tolist()
    assert st.tolist() == [0, 3]
    assert off == [0, len(want[0]), len(want[0]) + len(want[1])]
    assert np.array_equal(db.out[:len(want[0])].cpu().numpy(), want[0])


def test_device_batch_in_a_cuda_graph_reads_records_at_replay():
    """The whole call is recorded in a CUDA graph (no synchronisation or
    allocation inside it); rewriting the records on the device between
    replays changes the queries the graph runs."""
    T = skydata.mixed_table(50000, 12, 11)
    qa = skydata.batched_queries(128, T.shape[0], T.shape[1], seed=21, n_lo=50, n_hi=12000, d_lo=1, d_hi=12)
    qb = skydata.batched_queries(128, T.shape[0], T.shape[1], seed=22, n_lo=50, n_hi=12000, d_lo=1, d_hi=12)
    t = torch.from_numpy(T).cuda()
    bound = int(max(qa[:, 1].sum(), qb[:, 1].sum()))
    db = sky.DeviceBatch(t, 128, bound)
    rec = _records(qa)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        db.run(rec, stream=s)                    # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        db.run(rec, stream=torch.cuda.current_stream())
    for q in (qb, qa, qb):
        rec.copy_(_records(q))
        g.replay()
        got, st = db.results(), db.query_status()
        want, _ = _host(t, q)
        assert st.tolist() == [0] * len(q)
        for i in range(len(q)):
            assert np.array_equal(got[i], want[i]), i


def test_device_batch_workspace_too_small_is_refused():
    T = skydata.mixed_table(1000, 4, 1)
    t = torch.from_numpy(T).cuda()
    lib = sky._load_batched()
    need = lib.sky_batched_device_workspace_size(4, 2, 1000)
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    rec = _records(np.array([(0, 500, 0b11), (500, 500, 0b111)]))
    off = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    out = torch.empty(1000, dtype=torch.int32, device="cuda")
    args = [sky._vp(t.data_ptr()), 1000, 4, 4, 1, sky._vp(rec.data_ptr()), 2, 1000]
    rest = [sky._vp(out.data_ptr()), 1000, sky._vp(off.data_ptr()), sky._vp(st.data_ptr()), None]
    assert lib.sky_skyline_batched_device(*args, sky._vp(ws.data_ptr()), need - 256, *rest) == 3
    assert lib.sky_skyline_batched_device(*args, sky._vp(ws.data_ptr() + 8), need, *rest) == 1   # misaligned
    assert lib.sky_skyline_batched_device(*args, sky._vp(ws.data_ptr()), need, *rest) == 0
    torch.cuda.synchronize()
    assert st.tolist() == [0, 0]
