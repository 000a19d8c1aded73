"""Pins for the oracle's skyline (Definitions 1 and 2, SFS of Sec. 2.1).

Each check is fixed by the paper or by the mathematics, not by re-running the
oracle's own formula: Table 1's printed skyline, closed-form cases (d = 1,
anti-chains, duplicates), the two defining properties of a skyline, and
metamorphic identities. A dropped strictness test, a flipped comparison or a
wrong index in the oracle fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
import skydata


def test_table1_restaurants(golden):
    g = golden("table1_restaurants.json")
    P = np.array(g["points"], dtype=np.float32)
    assert oracle.skyline_brute(P).tolist() == g["skyline"]
    assert oracle.skyline_sfs(P).tolist() == g["skyline"]
    for i, j in g["dominated_by"].items():
        assert oracle.dominates(P[j], P[int(i)])
        assert oracle.dominator(P, int(i)) == j
    for i in g["skyline"]:
        assert oracle.dominator(P, i) == -1


def test_definition1_cases():
    # all <= and one <: dominates; equal: no; mixed: no; strictly: yes
    assert oracle.dominates([1, 2, 3], [1, 2, 4])
    assert not oracle.dominates([1, 2, 3], [1, 2, 3])
    assert not oracle.dominates([1, 2, 5], [1, 3, 4])
    assert oracle.dominates([0, 0], [1, 1])
    assert not oracle.dominates([1, 1], [0, 0])
    assert not oracle.dominates([1.0], [1.0])
    # -0.0 and +0.0 compare equal in IEEE arithmetic
    assert not oracle.dominates([-0.0, 1.0], [0.0, 1.0])


def test_d1_is_minimum():
    rng = np.random.default_rng(5)
    for _ in range(50):
        x = rng.integers(0, 6, size=rng.integers(1, 40)).astype(np.float32)
        want = np.flatnonzero(x == x.min()).tolist()
        assert oracle.skyline_brute(x).tolist() == want
        assert oracle.skyline_sfs(x).tolist() == want


def test_antichain_all_skyline():
    n = 500
    x0 = np.arange(n, dtype=np.float32)
    x1 = np.arange(n, dtype=np.float32)[::-1].copy()
    P = np.stack([x0, x1], axis=1)
    rng = np.random.default_rng(1)
    P = P[rng.permutation(n)]
    assert oracle.skyline_brute(P).tolist() == list(range(n))
    assert oracle.skyline_sfs(P).tolist() == list(range(n))


def test_integer_hyperplane_all_skyline():
    # every integer point with coordinates summing to K is incomparable with the others
    K, d = 6, 3
    pts = [p for p in itertools.product(range(K + 1), repeat=d) if sum(p) == K]
    P = np.array(pts, dtype=np.float32)
    assert oracle.skyline_sfs(P).size == len(pts)
    assert oracle.skyline_brute(P).size == len(pts)


def test_duplicates_kept_and_not_dominating():
    P = np.array([[0.5, 0.5], [0.5, 0.5], [0.6, 0.6], [0.5, 0.7]], dtype=np.float32)
    # the two copies do not dominate each other; both dominate the rest
    assert oracle.skyline_brute(P).tolist() == [0, 1]
    assert oracle.skyline_sfs(P).tolist() == [0, 1]


def _check_skyline_properties(P, S):
    n = P.shape[0]
    inS = np.zeros(n, bool)
    inS[S] = True
    for i in S:
        assert oracle.dominator(P, int(i)) == -1
    for i in np.flatnonzero(~inS):
        # some skyline point dominates every non-skyline point
        assert any(oracle.dominates(P[j], P[i]) for j in S)


@pytest.mark.parametrize("kind", ["independent", "correlated", "anticorrelated"])
@pytest.mark.parametrize("d", [2, 3, 5])
def test_skyline_properties(kind, d):
    P = skydata.generate(kind, 300, d, seed=11 + d)
    S = oracle.skyline_brute(P)
    assert S.size > 0
    _check_skyline_properties(P, S)


def test_brute_equals_sfs_random_small():
    """10^4 random small cases, heavy ties, d = 1..6, clipped 0/1 values."""
    rng = np.random.default_rng(123)
    for case in range(10000):
        n = int(rng.integers(0, 24))
        d = int(rng.integers(1, 7))
        mode = case % 4
        if mode == 0:
            P = rng.integers(0, 3, size=(n, d)).astype(np.float32) / 2
        elif mode == 1:
            P = rng.random((n, d), dtype=np.float32)
        elif mode == 2:
            P = np.clip(rng.normal(0.5, 0.6, size=(n, d)), 0, 1).astype(np.float32)
        else:
            P = rng.integers(-2, 2, size=(n, d)).astype(np.float32) * np.float32(1e30)
        a = oracle.skyline_brute(P, threads=1)
        b = oracle.skyline_sfs(P, threads=1)
        assert a.tolist() == b.tolist(), (case, n, d)


@pytest.mark.parametrize("kind", ["independent", "anticorrelated", "correlated"])
def test_brute_equals_sfs_medium(kind):
    P = skydata.generate(kind, 4000, 4, seed=3)
    assert oracle.skyline_brute(P).tolist() == oracle.skyline_sfs(P).tolist()


def test_metamorphic_permutations_and_transforms():
    rng = np.random.default_rng(9)
    P = skydata.generate("independent", 2000, 4, seed=9)
    S = oracle.skyline_sfs(P)
    # row permutation permutes the indices
    perm = rng.permutation(P.shape[0])
    S2 = oracle.skyline_sfs(P[perm])
    assert sorted(perm[S2].tolist()) == S.tolist()
    # dimension permutation leaves the set unchanged
    assert oracle.skyline_sfs(P[:, [2, 0, 3, 1]]).tolist() == S.tolist()
    # strictly increasing per-dimension transforms leave the set unchanged
    assert oracle.skyline_sfs(P * np.float32(8.0)).tolist() == S.tolist()
    # replacing every value by its rank within its dimension is strictly
    # increasing and exact in float32
    R = np.empty_like(P)
    for k in range(P.shape[1]):
        _, inv = np.unique(P[:, k], return_inverse=True)
        R[:, k] = inv.astype(np.float32)
    assert oracle.skyline_sfs(R).tolist() == S.tolist()
    # negating one dimension changes the problem: the set must differ here
    Nn = P.copy()
    Nn[:, 0] = -Nn[:, 0]
    assert oracle.skyline_sfs(Nn).tolist() != S.tolist()


def test_union_identity():
    P = skydata.generate("anticorrelated", 3000, 3, seed=4)
    A, B = P[:1700], P[1700:]
    SA = oracle.skyline_sfs(A)
    SB = oracle.skyline_sfs(B) + 1700
    cand = np.concatenate([SA, SB])
    Sc = cand[oracle.skyline_sfs(P[cand])]
    assert sorted(Sc.tolist()) == oracle.skyline_sfs(P).tolist()


def test_o5_cross_cell_domination():
    """Reading of the refinement step: a point in one candidate cell can be
    dominated by a point in another candidate cell (G = 4)."""
    P = np.array([[0.1, 0.55], [0.2, 0.8]], dtype=np.float32)
    keys = oracle.cell_keys(P, log2g=2, assume_unit=True)
    ca = oracle.cell_columns(keys[0], 2, 2)
    cb = oracle.cell_columns(keys[1], 2, 2)
    assert ca == (0, 2) and cb == (0, 3)
    occ = oracle.occupancy(keys, 2, 2)
    dom, key, cand, _ = oracle.cell_classes(occ, 2, 2)
    assert cand[keys[1]] and not dom[keys[1]]      # b's cell survives cell pruning
    assert oracle.skyline_brute(P).tolist() == [0]  # yet a dominates b


def test_quadrant_query_definition():
    """A quadrant query keeps the rows >= the origin in every selected column;
    its skyline equals the skyline of those rows shifted to the origin (the
    comparison of Definition 1 is translation invariant), and a row below the
    origin in one column never takes part, even when it would dominate."""
    rng = np.random.default_rng(31)
    T = rng.random((400, 5)).astype(np.float32)
    mask = 0b10110                                     # columns 1, 2, 4
    o = np.array([0.2, 0.35, 0.1], dtype=np.float32)
    got = oracle.skyline_subset(T, 50, 300, mask, origin=o)
    sub = T[50:350][:, [1, 2, 4]]
    inq = np.all(sub >= o, axis=1)
    shifted = (sub[inq] - o).astype(np.float32)
    brute = np.flatnonzero(inq)[oracle.skyline_brute(shifted)] + 50
    assert got.tolist() == brute.tolist()
    # a dominating row outside the quadrant is ignored
    U = np.array([[0.5, 0.5], [0.6, 0.6], [0.1, 0.9]], dtype=np.float32)
    assert oracle.skyline_subset(U, 0, 3, 0b11).tolist() == [0, 2]
    assert oracle.skyline_subset(U, 0, 3, 0b11, origin=[0.55, 0.0]).tolist() == [1]
    # an origin below every row changes nothing
    assert oracle.skyline_subset(T, 0, 400, mask, origin=[-1, -1, -1]).tolist() == \
        oracle.skyline_subset(T, 0, 400, mask).tolist()


def test_snap_rows_pins():
    """oracle.snap_rows: smallest binary32 sum among the points <= f, ties to
    the lower row, -1 without a candidate."""
    P = np.array([[0.5, 0.5], [0.2, 0.9], [0.9, 0.1], [0.3, 0.3]], dtype=np.float32)
    F = np.array([[0.6, 0.6], [0.1, 0.1], [1.0, 1.0], [0.9, 0.5]], dtype=np.float32)
    # f0: rows 0 (1.0) and 3 (0.6) qualify -> 3; f1: none; f2: all, 3 smallest;
    # f3: rows 0 (1.0), 2 (1.0), 3 (0.6) -> 3
    assert oracle.snap_rows(P, F).tolist() == [3, -1, 3, 3]
    # equal sums: the lower row
    Q = np.array([[0.2, 0.3], [0.3, 0.2]], dtype=np.float32)
    assert oracle.snap_rows(Q, [[1, 1]]).tolist() == [0]
    # the sum is binary32 in dimension order: 1 + 2^-24 + 2^-24 rounds to 1
    # (ties to even at each step), below 1 + 2^-23, although both are
    # 1 + 2^-23 in exact arithmetic (where the tie would pick row 0)
    e = np.float32(2.0 ** -24)
    R = np.array([[np.float32(1.0) + np.float32(2.0 ** -23), 0, 0], [1.0, e, e]], dtype=np.float32)
    assert oracle.snap_rows(R, [[2, 2, 2]]).tolist() == [1]
    # a point equal to f qualifies (<=, not <)
    assert oracle.snap_rows(P, [[0.9, 0.1]]).tolist() == [2]
