"""The paper's sequential SkyCell on the host (sky_baseline_sequential): the
CPU baseline the GPU path is timed against. Pinned to the oracle: the key
cells its slice enumeration finds are Definition 4's, and its skyline is the
oracle's, exactly. Host code only -- these tests need no GPU."""
import numpy as np
import pytest

import oracle
import skydata

sky = pytest.importorskip("paper_2107_09993_b300")


def test_table1_restaurants(golden):
    g = golden("table1_restaurants.json")
    P = np.array(g["points"], dtype=np.float32)
    got, _ = sky.baseline_sequential(P)
    assert got.tolist() == g["skyline"]


def test_key_cells_are_definition_4():
    """Layer by layer the slice enumeration (start bound doubled from the
    previous layer, end bound from the lower slices) yields exactly the
    non-empty cells no other non-empty cell is <= (the oracle's Def. 4)."""
    for trial in range(150):
        rng = np.random.default_rng(trial)
        d = int(rng.integers(1, 5))
        lg = int(rng.integers(1, 7))
        while lg * d > 12:
            lg -= 1
        n = int(rng.integers(1, 400))
        P = skydata.generate(["independent", "correlated", "anticorrelated"][trial % 3], n, d, seed=trial)
        keys = sky.baseline_key_cells(P, lg, assume_unit=True)
        occ = oracle.occupancy(oracle.cell_keys(P, lg, assume_unit=True), d, lg)
        _, key, _, _ = oracle.cell_classes(occ, d, lg)
        assert keys.tolist() == np.flatnonzero(key).tolist(), (trial, d, lg, n)


def test_candidates_are_the_points_of_non_dominated_cells():
    for i, (kind, n, d, lg) in enumerate([("independent", 3000, 3, 3), ("correlated", 4000, 2, 5),
                                          ("anticorrelated", 2000, 4, 2)]):
        P = skydata.generate(kind, n, d, seed=30 + i)
        _, cand = sky.baseline_sequential(P, log2_g=lg, assume_unit=True)
        keys = oracle.cell_keys(P, lg, assume_unit=True)
        dom, _, _, _ = oracle.cell_classes(oracle.occupancy(keys, d, lg), d, lg)
        assert cand == int((dom[keys.astype(np.int64)] == 0).sum())


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 12, 16])
@pytest.mark.parametrize("kind", ["independent", "correlated", "anticorrelated"])
def test_skyline_equals_oracle(kind, d):
    n = 3000 if d <= 8 else 800
    P = skydata.generate(kind, n, d, seed=200 + d)
    got, cand = sky.baseline_sequential(P)
    want = oracle.skyline_brute(P)
    assert got.tolist() == want.tolist()
    assert cand >= got.size


def test_ties_duplicates_and_values_outside_the_unit_cube():
    rng = np.random.default_rng(7)
    P = rng.integers(0, 4, size=(2000, 4)).astype(np.float32)   # heavy ties and duplicates
    P[100:110] = P[0]
    want = oracle.skyline_brute(P).tolist()
    for lg in (None, 1, 3, 6):
        assert sky.baseline_sequential(P, log2_g=lg)[0].tolist() == want
    Q = (skydata.anticorrelated(1500, 3, seed=8) * 1e6 - 5e5).astype(np.float32)
    assert sky.baseline_sequential(Q)[0].tolist() == oracle.skyline_brute(Q).tolist()


def test_errors():
    P = skydata.independent(10, 3, seed=1)
    P[4, 1] = np.nan
    with pytest.raises(sky.SkyError) as e:
        sky.baseline_sequential(P)
    assert e.value.name == "SKY_ERR_NONFINITE"
    with pytest.raises(sky.SkyError) as e:
        sky.baseline_sequential(skydata.independent(10, 8, seed=1), log2_g=4)
    assert e.value.name == "SKY_ERR_TOO_LARGE"
    assert sky.baseline_sequential(np.zeros((0, 3), dtype=np.float32))[0].size == 0
