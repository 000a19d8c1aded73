"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The skyline is a set with a canonical (ascending) order, so every comparison
here is exact equality of int32 index arrays -- never a tolerance.
"""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_sky(P, **kw):
    return sky.skyline(dev(P), **kw).cpu().numpy().tolist()


def test_table1_restaurants(golden):
    g = golden("table1_restaurants.json")
    P = np.array(g["points"], dtype=np.float32)
    assert gpu_sky(P) == g["skyline"]


def test_config0_uniform_20000x4():
    """n = 20,000, d = 4, independent uniform [0,1), seed 0 (brute force oracle)."""
    P = skydata.independent(20000, 4, seed=0)
    want = oracle.skyline_brute(P).tolist()
    assert gpu_sky(P) == want
    assert gpu_sky(P, assume_unit=True) == want
    for lg in (0, 1, 3, 6):
        assert gpu_sky(P, log2_g=lg, assume_unit=True) == want


SIZES = [1, 2, 3, 31, 127, 128, 129, 255, 256, 257, 2047, 2048, 2049, 4097, 9001]


@pytest.mark.parametrize("n", SIZES)
def test_ragged_sizes(n):
    rng = np.random.default_rng(n)
    d = int(rng.integers(1, 17))
    P = skydata.anticorrelated(n, d, seed=n)
    want = oracle.skyline_sfs(P).tolist()
    assert gpu_sky(P) == want
    assert gpu_sky(P, assume_unit=True) == want


@pytest.mark.parametrize("d", list(range(1, 17)))
@pytest.mark.parametrize("kind", ["independent", "correlated", "anticorrelated"])
def test_every_dimension(kind, d):
    n = 3000 if d <= 8 else 1500
    P = skydata.generate(kind, n, d, seed=100 + d)
    want = oracle.skyline_sfs(P).tolist()
    assert gpu_sky(P) == want
    assert gpu_sky(P, assume_unit=True) == want


def test_heavy_ties_duplicates_and_clipping():
    rng = np.random.default_rng(7)
    for case in range(40):
        n = int(rng.integers(1, 3000))
        d = int(rng.integers(1, 9))
        levels = int(rng.integers(2, 6))
        P = (rng.integers(0, levels, size=(n, d)) / (levels - 1)).astype(np.float32)
        P[: n // 3] = P[0]                              # many exact duplicates
        want = oracle.skyline_sfs(P).tolist()
        assert gpu_sky(P) == want, case
        assert gpu_sky(P, assume_unit=True) == want, case


def test_general_values_outside_unit_cube():
    rng = np.random.default_rng(8)
    P = (rng.standard_normal((5000, 5)) * np.array([1e-3, 1, 50, 1e6, 3])).astype(np.float32)
    P[:, 4] = -2.5                                      # a constant dimension
    P[17] = -0.0
    want = oracle.skyline_sfs(P).tolist()
    assert gpu_sky(P) == want
    # the unit-cube map clamps: still exact
    assert gpu_sky(P, assume_unit=True) == want


def test_strided_and_unaligned_rows():
    rng = np.random.default_rng(9)
    base = rng.random((4000, 11), dtype=np.float32)
    want = oracle.skyline_sfs(np.ascontiguousarray(base[:, :7])).tolist()
    t = torch.from_numpy(base).cuda()
    assert sky.skyline(t[:, :7]).cpu().tolist() == want            # ld = 11 > d = 7
    flat = torch.zeros(4000 * 8 + 1, dtype=torch.float32, device="cuda")
    P8 = rng.random((4000, 8), dtype=np.float32)
    flat[1:].copy_(torch.from_numpy(P8.ravel()))
    un = flat[1:].view(4000, 8)                                     # 4-byte, not 16-byte aligned
    assert sky.skyline(un).cpu().tolist() == oracle.skyline_sfs(P8).tolist()


def test_filter_proposals_never_change_the_result():
    rng = np.random.default_rng(10)
    for kind in ("independent", "correlated", "anticorrelated"):
        P = skydata.generate(kind, 20000, 6, seed=11)
        want = oracle.skyline_sfs(P).tolist()
        prop = dev(rng.random((16, 6)).astype(np.float32) * 0.6)
        assert sky.skyline(dev(P), filter_points=prop).cpu().tolist() == want
        st = sky.last_run_stats()
        assert 0 <= st["n_filter_used"] <= 16
        # proposals below every point snap to nothing and are dropped
        low = dev(np.full((4, 6), -1.0, dtype=np.float32))
        assert sky.skyline(dev(P), filter_points=low).cpu().tolist() == want
        assert sky.last_run_stats()["n_filter_used"] == 0


def test_snapped_rows_match_oracle():
    """The pre-filter's snap (k_snap) picks, per proposal, the row that the
    oracle's restatement picks: among the points <= f, the smallest binary32
    coordinate sum, ties to the lower row; -1 without a candidate. Includes
    many equal sums (integer grids) and proposals below every point."""
    rng = np.random.default_rng(21)
    for case in range(12):
        d = int(rng.integers(1, 17))
        n = int(rng.integers(1, 30000))
        if case % 3 == 2:
            P = rng.integers(0, 4, size=(n, d)).astype(np.float32)          # heavy ties
            F = rng.integers(0, 4, size=(16, d)).astype(np.float32)
        else:
            P = skydata.generate(["independent", "anticorrelated"][case % 2], n, d, seed=case)
            F = (rng.random((16, d)) * 0.9).astype(np.float32)
        F[3] = -1.0                                                             # snaps to nothing
        g = sky.Grid(dev(P)).prune(dev(F))
        got = g.snap_rows(16)
        want = oracle.snap_rows(P, F).tolist()
        assert got == want, (case, n, d)
        assert g.stats()["n_filter_used"] == sum(w >= 0 for w in want)
        g.close()


def test_cell_grid_matches_oracle():
    """Steps (a)-(c) bit for bit: keys (Eq. 1), occupancy, dominated cells (Def. 3)."""
    rng = np.random.default_rng(12)
    for case in range(30):
        d = int(rng.integers(1, 5))
        lg = int(rng.integers(0, {1: 8, 2: 6, 3: 4, 4: 3}[d]))
        n = int(rng.integers(1, 4000))
        kind = ["independent", "correlated", "anticorrelated"][case % 3]
        P = skydata.generate(kind, n, d, seed=case)
        mode = ["auto", "unit", "minmax"][case % 3 if case % 4 else 1]
        if case % 5 == 0:
            P = (P * np.float32(0.3) + np.float32(0.1)).astype(np.float32)   # narrow range: auto normalises
        g = sky.Grid(dev(P), log2_g=lg, assume_unit={"auto": 0, "unit": 1, "minmax": 2}[mode]).prune()
        keys = g.cell_keys().cpu().numpy().view(np.uint32).astype(np.uint64)
        want_keys = oracle.cell_keys(P, lg, mode=mode)
        assert np.array_equal(keys, want_keys), case
        ncell = 1 << (lg * d)
        occ_bits = np.unpackbits(g.occupied().cpu().numpy().view(np.uint8), bitorder="little")[:ncell]
        assert np.array_equal(occ_bits, oracle.occupancy(want_keys, d, lg)), case
        dom_bits = np.unpackbits(g.dominated().cpu().numpy().view(np.uint8), bitorder="little")[:ncell]
        if ncell <= 4096:
            dom, key, cand, ncand = oracle.cell_classes(oracle.occupancy(want_keys, d, lg), d, lg)
            assert np.array_equal(dom_bits, dom), case
        surv = g.survivors().cpu().numpy()
        assert surv.tolist() == np.flatnonzero(dom_bits[want_keys.astype(np.int64)] == 0).tolist()
        st = g.stats()
        assert st["occupied_cells"] == int(occ_bits.sum())
        # soundness: every skyline point survives step (c)
        S = oracle.skyline_sfs(P)
        assert set(S.tolist()) <= set(surv.tolist())
        g.close()


@pytest.mark.parametrize("d,lg", [(2, 9), (2, 12), (2, 13), (3, 6), (3, 8), (3, 9), (4, 5), (4, 6), (5, 5),
                                  (6, 4), (7, 3), (8, 3), (9, 3), (10, 2), (12, 2), (13, 2), (16, 1)])
def test_large_grid_prefix_matches_oracle(d, lg):
    """Grids of 2^16 .. 2^27 cells, where the prefix-OR splits into blocks
    of low dimensions and rows of high dimensions: the dominated bitmap and
    the survivors equal Definition 3 computed by the oracle's box identity."""
    rng = np.random.default_rng(d * 100 + lg)
    n = 6000
    kind = ["independent", "correlated", "anticorrelated"][(d + lg) % 3]
    P = skydata.generate(kind, n, d, seed=d + lg)
    # a few points near the low corner and clusters make long dominated runs
    P[:50] = (rng.random((50, d)) * 0.2).astype(np.float32)
    g = sky.Grid(dev(P), log2_g=lg, assume_unit=True).prune()
    want_keys = oracle.cell_keys(P, lg, assume_unit=True)
    keys = g.cell_keys().cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(keys, want_keys)
    ncell = 1 << (lg * d)
    occ = oracle.occupancy(want_keys, d, lg)
    want_dom = oracle.dominated_cells(occ, d, lg)
    dom_bits = np.unpackbits(g.dominated().cpu().numpy().view(np.uint8), bitorder="little")[:ncell]
    assert np.array_equal(dom_bits, want_dom)
    surv = g.survivors().cpu().numpy()
    assert surv.tolist() == np.flatnonzero(want_dom[want_keys.astype(np.int64)] == 0).tolist()
    g.close()
    # the full path on the same grid returns the exact skyline
    assert gpu_sky(P, log2_g=lg, assume_unit=True) == oracle.skyline_sfs(P).tolist()


def test_survivors_only_returns_step_c_candidates():
    """survivors_only stops after step (c): the rows whose cell no occupied
    cell dominates (Definition 3, the oracle's box identity on the oracle's
    cell keys), ascending; a superset of the skyline."""
    for i, (kind, n, d) in enumerate([("independent", 50000, 4), ("correlated", 120000, 6),
                                      ("anticorrelated", 30000, 3), ("independent", 300000, 8)]):
        P = skydata.generate(kind, n, d, seed=40 + i)
        x = dev(P)
        got = sky.skyline(x, survivors_only=True).cpu().numpy()
        lg = sky.last_run_stats()["log2_g"]
        keys = oracle.cell_keys(P, lg, mode="auto")
        dom = oracle.dominated_cells(oracle.occupancy(keys, d, lg), d, lg)
        want = np.flatnonzero(dom[keys.astype(np.int64)] == 0)
        assert got.tolist() == want.tolist(), (kind, n, d)
        assert set(oracle.skyline_sfs(P).tolist()) <= set(got.tolist())
        # a buffer shorter than n takes the copy path; same ids
        got2 = sky.skyline(x, survivors_only=True, capacity=len(want)).cpu().numpy()
        assert got2.tolist() == want.tolist()
        with pytest.raises(sky.SkyError) as e:
            sky.skyline(x, survivors_only=True, capacity=len(want) - 1)
        assert e.value.name == "SKY_ERR_CAPACITY"


def test_device_timing_modes():
    """Mode 1 times the phases (kernels launched one by one), mode 2 the whole
    kernel sequence of a call (graph replay kept); neither changes the result,
    and other modes are rejected."""
    P = skydata.generate("independent", 200000, 6, seed=9)
    x = dev(P)
    want = gpu_sky(P)
    try:
        for mode in (1, 2):
            sky.set_phase_timing(mode)
            for _ in range(3):   # first call direct, later calls replay the captured graph
                assert sky.skyline(x).cpu().numpy().tolist() == want
                t = sky.last_phase_times()
                if mode == 1:
                    assert t["map_mark_ms"] > 0 and t["refine_ms"] > 0 and t["call_ms"] == 0
                else:
                    assert t["call_ms"] > 0 and t["map_mark_ms"] == 0
        with pytest.raises(sky.SkyError) as e:
            sky.set_phase_timing(3)
        assert e.value.name == "SKY_ERR_INVALID_ARGUMENT"
    finally:
        sky.set_phase_timing(False)


def test_fig1_and_fig2_dominated_cells(golden):
    g1 = golden("fig1_layer4.json")
    G = 1 << g1["log2g"]
    cells = [(c0, c1) for c1, c0 in g1["key_cells_c1_c0"]]
    P = np.array([[(c0 + 0.5) / G, (c1 + 0.5) / G] for c0, c1 in cells], dtype=np.float32)
    g = sky.Grid(dev(P), log2_g=g1["log2g"], assume_unit=True).prune()
    dom = np.unpackbits(g.dominated().cpu().numpy().view(np.uint8), bitorder="little")
    c1, c0 = g1["dominated_example_c1_c0"]
    assert dom[oracle.cell_key((c0, c1), 4)] == 1
    i1, i0 = g1["irrelevant_example_c1_c0"]
    assert dom[oracle.cell_key((i0, i1), 4)] == 0
    assert g.stats()["surviving_cells"] == 4          # the four key cells
    g2 = golden("fig2_layer2_3d.json")
    cells = [tuple(reversed(c)) for c in g2["occupied_cl2_cl1_cl0"]]
    P = np.array([[(c + 0.5) / 4 for c in cell] for cell in cells], dtype=np.float32)
    g = sky.Grid(dev(P), log2_g=2, assume_unit=True).prune()
    assert g.stats()["surviving_cells"] == 4
    assert gpu_sky(P) == [0, 1, 2, 3]


def test_errors():
    P = skydata.independent(1000, 3, seed=1)
    bad = P.copy()
    bad[500, 1] = np.nan
    with pytest.raises(sky.SkyError) as e:
        sky.skyline(dev(bad))
    assert e.value.name == "SKY_ERR_NONFINITE"
    bad[500, 1] = np.inf
    with pytest.raises(sky.SkyError) as e:
        sky.skyline(dev(bad), assume_unit=True)
    assert e.value.name == "SKY_ERR_NONFINITE"
    want = oracle.skyline_sfs(P)
    with pytest.raises(sky.SkyError) as e:
        sky.skyline(dev(P), capacity=len(want) - 1)
    assert e.value.name == "SKY_ERR_CAPACITY" and f"count={len(want)}" in str(e.value)
    assert sky.skyline(dev(P), capacity=len(want)).cpu().tolist() == want.tolist()
    with pytest.raises(sky.SkyError) as e:
        sky.skyline(dev(P), log2_g=10)
    assert e.value.name == "SKY_ERR_TOO_LARGE"
    with pytest.raises(sky.SkyError) as e:
        sky.skyline(dev(np.zeros((10, 17), np.float32)))
    assert e.value.name == "SKY_ERR_INVALID_ARGUMENT"
    assert sky.skyline(torch.empty((0, 3), dtype=torch.float32, device="cuda")).numel() == 0


def test_host_entry_point():
    P = skydata.anticorrelated(30000, 5, seed=2)
    want = oracle.skyline_sfs(P).tolist()
    h = torch.from_numpy(P).pin_memory()
    assert sky.skyline_host(h).tolist() == want
    assert sky.skyline_host(torch.from_numpy(P)).tolist() == want


def test_repeat_is_deterministic():
    P = dev(skydata.anticorrelated(200000, 8, seed=3))
    a = sky.skyline(P).cpu()
    s1 = sky.last_run_stats()
    b = sky.skyline(P).cpu()
    s2 = sky.last_run_stats()
    assert torch.equal(a, b)
    assert s1["survivors"] == s2["survivors"] and s1["skyline"] == s2["skyline"] == a.numel()
