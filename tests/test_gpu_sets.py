"""Parity of the multi-set entry points (sky_skyline_sets,
sky_skyline_host_sets) with the CPU oracle, set by set: exact equality of
the ascending index arrays. Covers mixed d and distributions, an empty set,
more sets than concurrent slots, repeated calls (graph replay), per-set
capacity failures and the summed run counters."""
import ctypes

import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def mixed_sets():
    specs = [("independent", 9001, 3, 1), ("anticorrelated", 5000, 8, 2), ("correlated", 20000, 5, 3),
             ("anticorrelated", 129, 16, 4), ("independent", 0, 4, 5), ("anticorrelated", 3000, 2, 6),
             ("independent", 4097, 12, 7)]
    out = []
    for kind, n, d, seed in specs:
        P = skydata.generate(kind, n, d, seed) if n else np.zeros((0, d), np.float32)
        out.append(np.ascontiguousarray(P, dtype=np.float32))
    return out


@pytest.fixture(scope="module")
def sets_and_want():
    sets = mixed_sets()
    want = [oracle.skyline_sfs(P).tolist() if len(P) else [] for P in sets]
    return sets, want


def test_device_sets_match_oracle(sets_and_want):
    sets, want = sets_and_want
    xs = [torch.from_numpy(P).cuda() for P in sets]
    for _ in range(3):   # first call direct, then captured, then replayed
        got = sky.skyline_sets(xs)
        assert [g.cpu().tolist() for g in got] == want
    st = sky.last_run_stats()
    assert st["n"] == sum(len(P) for P in sets)
    assert st["skyline"] == sum(len(w) for w in want)
    assert st["kernels"] > 0


def test_host_sets_match_oracle(sets_and_want):
    sets, want = sets_and_want
    pinned = [torch.from_numpy(P).pin_memory() for P in sets]
    pageable = [torch.from_numpy(P.copy()) for P in sets]
    for src in (pinned, pageable, pinned):
        got = sky.skyline_host_sets(src)
        assert [g.tolist() for g in got] == want


def test_sets_equal_single_calls_with_options(sets_and_want):
    sets, _ = sets_and_want
    xs = [torch.from_numpy(P).cuda() for P in sets if len(P)]
    for kw in ({"assume_unit": True}, {"log2_g": 1, "assume_unit": 2}, {"survivors_only": True}):
        one = [sky.skyline(x, **kw).cpu().tolist() for x in xs]
        for _ in range(2):
            assert [g.cpu().tolist() for g in sky.skyline_sets(xs, **kw)] == one


@pytest.mark.parametrize("host", [False, True])
def test_capacity_failure_is_per_set(host):
    lib = sky.load()
    Ps = [np.ascontiguousarray(skydata.generate("anticorrelated", 3000, 6, s), dtype=np.float32) for s in (1, 2, 3)]
    want = [oracle.skyline_sfs(P).tolist() for P in Ps]
    caps = [3000, 5, 3000]
    if host:
        src = [torch.from_numpy(P).pin_memory() for P in Ps]
        outs = [torch.full((c,), -7, dtype=torch.int32).pin_memory() for c in caps]
    else:
        src = [torch.from_numpy(P).cuda() for P in Ps]
        outs = [torch.full((c,), -7, dtype=torch.int32, device="cuda") for c in caps]
    arr = (sky.SkySet * 3)()
    for i in range(3):
        arr[i].pts, arr[i].n, arr[i].d, arr[i].ld = src[i].data_ptr(), 3000, 6, 6
        arr[i].out_idx, arr[i].capacity = outs[i].data_ptr(), caps[i]
    fn = lib.sky_skyline_host_sets if host else lib.sky_skyline_sets
    st = fn(arr, 3, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 3 and lib.sky_last_error().startswith(b"set 1:")
    assert [a.status for a in arr] == [0, 3, 0]
    assert arr[1].count == len(want[1]) > 5
    for i in (0, 2):
        assert outs[i][:arr[i].count].cpu().tolist() == want[i]
    if host:   # the first `capacity` ids still arrive
        assert outs[1].tolist() == want[1][:5]


def test_nonfinite_set_fails_alone():
    Ps = [np.ascontiguousarray(skydata.generate("independent", 2000, 4, s), dtype=np.float32) for s in (1, 2)]
    bad = Ps[1].copy()
    bad[17, 2] = np.nan
    xs = [torch.from_numpy(Ps[0]).cuda(), torch.from_numpy(bad).cuda()]
    with pytest.raises(sky.SkyError) as e:
        sky.skyline_sets(xs)
    assert e.value.status == 2
    assert "set 1" in str(e.value)
