"""Witness mode (sky_skyline_witness) against the oracle.

For every input here the oracle's skyline is known exactly, so the test checks
both directions: the witness call returns the oracle's index set, every
returned row carries -1, and every other row carries a point that dominates it
(Definition 1). The cases reach each of the three places a point can be
dropped: a dominated cell (step c; forced fine layers make many), a snapped
proposal (step c'), and the refinement (step d)."""
import numpy as np
import pytest

import oracle
import skydata
from parity import check_witnesses

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run(P, **kw):
    S, W = sky.skyline_witness(dev(P), **kw)
    return S.cpu().numpy(), W.cpu().numpy()


def test_table1_witnesses(golden):
    g = golden("table1_restaurants.json")
    P = np.array(g["points"], dtype=np.float32)
    S, W = run(P)
    assert S.tolist() == g["skyline"]
    # r1 and r3 are both dominated by r2 only (Table 1)
    assert W.tolist() == [1, -1, 1, -1]


@pytest.mark.parametrize("kind", ["independent", "correlated", "anticorrelated"])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 12, 16])
def test_witnesses_match_oracle(kind, d):
    n = 5000 if d <= 8 else 2500
    P = skydata.generate(kind, n, d, seed=300 + d)
    want = oracle.skyline_sfs(P)
    S, W = run(P)
    assert np.array_equal(S, want)
    check_witnesses(P, S, W)
    # the witness mode returns what the plain entry point returns
    assert np.array_equal(sky.skyline(dev(P)).cpu().numpy(), want)


@pytest.mark.parametrize("log2_g", [1, 2, 3, 5])
def test_cell_witnesses_at_forced_layers(log2_g):
    """Fine layers on the unit-cube map drop most points at step (c); each of
    them needs a point of a lower occupied cell as witness."""
    d = 4
    P = skydata.independent(20000, d, seed=log2_g)
    want = oracle.skyline_sfs(P)
    S, W = run(P, log2_g=log2_g, assume_unit=True)
    assert np.array_equal(S, want)
    n_drop = check_witnesses(P, S, W)
    assert n_drop == P.shape[0] - want.size


def test_proposal_witnesses():
    """Proposals snapped to real rows remove points before step (d); their
    witness is the snapped row."""
    P = skydata.correlated(40000, 6, seed=9)
    want = oracle.skyline_sfs(P)
    rng = np.random.default_rng(1)
    F = np.clip(np.quantile(P, 0.3, axis=0) + rng.normal(0, 0.05, size=(16, 6)), 0, 1).astype(np.float32)
    S, W = run(P, log2_g=0, filter_points=dev(F))
    assert np.array_equal(S, want)
    check_witnesses(P, S, W)


def test_ties_and_duplicates():
    """Repeated rows are kept together; equal coordinates need the exact test."""
    rng = np.random.default_rng(5)
    base = rng.integers(0, 6, size=(3000, 5)).astype(np.float32)
    P = np.concatenate([base, base[:700]])
    want = oracle.skyline_sfs(P)
    for kw in ({}, {"assume_unit": 2}, {"log2_g": 2, "assume_unit": 2}):
        S, W = run(P, **kw)
        assert np.array_equal(S, want), kw
        check_witnesses(P, S, W)


def test_witness_mode_rejects_survivors_only():
    x = dev(skydata.independent(100, 3, seed=0))
    W = torch.empty(100, dtype=torch.int32, device="cuda")
    out = torch.empty(100, dtype=torch.int32, device="cuda")
    import ctypes
    o = sky._opts(None, False, None, survivors_only=True)
    cnt = ctypes.c_int64(0)
    st = sky.load().sky_skyline_witness(ctypes.c_void_p(x.data_ptr()), 100, 3, 3, ctypes.byref(o),
                                        ctypes.c_void_p(out.data_ptr()), 100, ctypes.byref(cnt),
                                        ctypes.c_void_p(W.data_ptr()), None)
    assert st == 1
