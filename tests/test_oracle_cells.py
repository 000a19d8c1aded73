"""Pins for the oracle's grid (Eq. 1) and cell classes (Definitions 3-6).

Fixed points: the Eq. 1 example, the Fig. 1 and Fig. 2 reconstructions and the
Theorem 1 worked example (Psi / Theta), Corollary 1's count for any occupancy,
the printed counts (1, 3, 7, 15, 31; 15 of 64; 63 of 1024; 28 leaves in Fig. 3),
Corollaries 3 and 4 across layers, and soundness of cell pruning against the
oracle's skyline.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import skydata


def cand_count(G, d):
    return G ** d - (G - 1) ** d


# ---------------------------------------------------------------- Eq. 1 ---

def test_eq1_worked_example(golden):
    g = golden("eq1_cell_example.json")
    P = np.array([[g["point_dim0"], g["point_dim1"]]], dtype=np.float32)
    for lay in g["layers"]:
        key = oracle.cell_keys(P, lay["layer"], assume_unit=True)[0]
        c0, c1 = oracle.cell_columns(key, 2, lay["layer"])
        assert (c1, c0) == (lay["col_dim1"], lay["col_dim0"])


def test_eq1_unit_cube_is_exact_floor():
    rng = np.random.default_rng(2)
    x = rng.random((2000, 3), dtype=np.float32)
    x[:5] = 0.0
    x[5:10] = np.float32(np.nextafter(np.float32(1), np.float32(0)))
    x[10:15] = 1.0           # outside [0,1): clamps to the last column
    for log2g in (1, 3, 6):
        G = 1 << log2g
        keys = oracle.cell_keys(x, log2g, assume_unit=True)
        for i in range(0, 2000, 7):
            cols = oracle.cell_columns(keys[i], 3, log2g)
            for k in range(3):
                want = min(int(Fraction(float(x[i, k])) * G), G - 1)
                assert cols[k] == want


def test_normalised_map_properties():
    rng = np.random.default_rng(4)
    P = (rng.random((3000, 4)) * np.array([5, 1e-3, 1e6, 1]) - 2).astype(np.float32)
    P[:, 3] = 7.0                                       # constant dimension
    log2g = 5
    G = 1 << log2g
    keys = oracle.cell_keys(P, log2g)
    cols = np.array([oracle.cell_columns(k, 4, log2g) for k in keys])
    for k in range(3):
        order = np.argsort(P[:, k], kind="stable")
        assert np.all(np.diff(cols[order, k]) >= 0)     # monotone
        assert cols[np.argmin(P[:, k]), k] == 0          # min -> first column
        assert cols[np.argmax(P[:, k]), k] == G - 1      # max -> last column
        assert len(np.unique(cols[:, k])) > G // 2       # uses the grid
    assert np.all(cols[:, 3] == 0)                       # zero range -> column 0


def test_automatic_map_choice():
    """The automatic map is Eq. 1 for data spanning most of the unit cube and
    the min/max normalisation otherwise (reading of Eq. 1 for general data)."""
    rng = np.random.default_rng(5)
    wide = rng.random((500, 3), dtype=np.float32)
    wide[0] = 0.0
    wide[1] = 1.0
    assert np.array_equal(oracle.cell_keys(wide, 4, mode="auto"), oracle.cell_keys(wide, 4, mode="unit"))
    narrow = (0.25 + 0.2 * rng.random((500, 3))).astype(np.float32)   # spans < 0.5
    assert np.array_equal(oracle.cell_keys(narrow, 4, mode="auto"), oracle.cell_keys(narrow, 4, mode="minmax"))
    assert not np.array_equal(oracle.cell_keys(narrow, 4, mode="auto"), oracle.cell_keys(narrow, 4, mode="unit"))
    neg = wide.copy()
    neg[7, 2] = -0.01                                                    # leaves [0, 1]
    assert np.array_equal(oracle.cell_keys(neg, 4, mode="auto"), oracle.cell_keys(neg, 4, mode="minmax"))
    big = wide.copy()
    big[9, 0] = 1.5
    assert np.array_equal(oracle.cell_keys(big, 4, mode="auto"), oracle.cell_keys(big, 4, mode="minmax"))
    # under min/max normalisation the extremes land in the first / last column
    cols = np.array([oracle.cell_columns(k, 3, 4) for k in oracle.cell_keys(narrow, 4, mode="minmax")])
    for k in range(3):
        assert cols[np.argmin(narrow[:, k]), k] == 0 and cols[np.argmax(narrow[:, k]), k] == 15


def test_automatic_map_decides_on_a_strided_sample():
    """Above 4096 rows the automatic map looks at rows 0, t, 2t, ... with
    t = ceil(n / 4096) only. An outlier off the sample leaves Eq. 1 in place
    (it is clamped into an edge column); on the sample it switches to the
    sample's min / max. Either way the map is monotone in every dimension."""
    rng = np.random.default_rng(9)
    n = 10_000                                   # t = 3
    P = rng.random((n, 3), dtype=np.float32)
    P[0] = 0.0
    P[3] = 0.999
    off_row = P.copy()
    off_row[3 * 1000 + 1, 1] = 7.0               # not a multiple of 3
    assert np.array_equal(oracle.cell_keys(off_row, 4, mode="auto"), oracle.cell_keys(off_row, 4, mode="unit"))
    assert oracle.cell_columns(int(oracle.cell_keys(off_row, 4, mode="auto")[3001]), 3, 4)[1] == 15
    on_row = P.copy()
    on_row[3 * 1000, 1] = 7.0                    # a sampled row
    off, sc = oracle.cell_params(on_row, 4, mode="auto")
    S = on_row[::3]
    assert np.array_equal(off, S.min(axis=0))
    assert np.array_equal(sc, (np.float32(16) / (S.max(axis=0) - S.min(axis=0))).astype(np.float32))
    # rows below the sample's minimum fall into column 0
    low = on_row.copy()
    low[5, 0] = -3.0
    keys = oracle.cell_keys(low, 4, mode="auto")
    assert oracle.cell_columns(int(keys[5]), 3, 4)[0] == 0
    # monotone: a componentwise smaller point never gets a larger column
    for Q in (off_row, on_row, low):
        cols = np.array([oracle.cell_columns(int(k), 3, 4) for k in oracle.cell_keys(Q, 4, mode="auto")])
        for k in range(3):
            o = np.argsort(Q[:, k], kind="stable")
            assert np.all(np.diff(cols[o, k]) >= 0)


# ---------------------------------------------------------- Definitions ---

def _occ_from_cells(cells_c0_first, d, log2g):
    occ = np.zeros(1 << (log2g * d), dtype=np.uint8)
    for c in cells_c0_first:
        occ[oracle.cell_key(c, log2g)] = 1
    return occ


def test_fig1_layer4(golden):
    g = golden("fig1_layer4.json")
    d, L = g["d"], g["log2g"]
    G = 1 << L
    key_cells = [(c0, c1) for c1, c0 in g["key_cells_c1_c0"]]
    # one point at the centre of each key cell
    P = np.array([[(c0 + 0.5) / G, (c1 + 0.5) / G] for c0, c1 in key_cells], dtype=np.float32)
    keys = oracle.cell_keys(P, L, assume_unit=True)
    occ = oracle.occupancy(keys, d, L)
    dom, key, cand, n_cand = oracle.cell_classes(occ, d, L)
    assert sorted(np.flatnonzero(key).tolist()) == sorted(oracle.cell_key(c, L) for c in key_cells)
    assert n_cand == g["n_candidates"] == cand_count(G, d)
    c1, c0 = g["dominated_example_c1_c0"]
    assert dom[oracle.cell_key((c0, c1), L)]
    b1, b0 = g["dominated_example_by_c1_c0"]
    assert b0 < c0 and b1 < c1 and occ[oracle.cell_key((b0, b1), L)]
    i1, i0 = g["irrelevant_example_c1_c0"]
    ik = oracle.cell_key((i0, i1), L)
    assert not dom[ik] and not cand[ik] and not occ[ik]
    # Theorem 1 worked example: Psi(L4[4,6]) = L4[4,15], Theta inverse with Phi = 6
    ps = g["psi_example"]
    cell = tuple(reversed(ps["cell_c1_c0"]))
    assert cand[oracle.cell_key(cell, L)]
    assert _Omega(cell, key, d, L) == ps["omega_cell"]
    assert _Psi(cell, key, d, L) == tuple(reversed(ps["image_c1_c0"]))
    th = g["theta_example"]
    ca = tuple(reversed(th["aux_cell_c1_c0"]))
    assert _gamma(ca, G) == th["gamma"]
    assert _Phi(ca, key, d, L) == th["phi"]
    assert _Theta(ca, key, d, L) == tuple(reversed(th["image_c1_c0"]))


def test_fig2_layer2_3d(golden):
    g = golden("fig2_layer2_3d.json")
    d, L = g["d"], g["log2g"]
    occ_cells = [tuple(reversed(c)) for c in g["occupied_cl2_cl1_cl0"]]
    occ = _occ_from_cells(occ_cells, d, L)
    dom, key, cand, n_cand = oracle.cell_classes(occ, d, L)
    want_keys = sorted(oracle.cell_key(tuple(reversed(c)), L) for c in g["key_cells_cl2_cl1_cl0"])
    assert sorted(np.flatnonzero(key).tolist()) == want_keys
    assert n_cand == g["n_candidates"]
    assert not dom[np.flatnonzero(occ)].any()


def test_corollary1_printed_counts(golden):
    g = golden("corollary1_counts.json")
    rng = np.random.default_rng(0)
    for L, want in enumerate(g["d2_layers_0_to_4"]):
        occ = (rng.random(1 << (2 * L)) < 0.1).astype(np.uint8)
        assert oracle.cell_classes(occ, 2, L)[3] == want
    occ = (rng.random(64) < 0.2).astype(np.uint8)
    assert oracle.cell_classes(occ, 2, 3)[3] == g["grid_8x8"]
    occ = (rng.random(1024) < 0.05).astype(np.uint8)
    assert oracle.cell_classes(occ, 2, 5)[3] == g["grid_32x32"]
    f = g["fig3_leaves"]
    assert (1 << f["d"]) * cand_count(1 << f["layer"], f["d"]) == f["leaves"]


def test_corollary1_any_occupancy():
    """|C_i| = G^d - (G-1)^d whatever the data (Theorem 1 + Lemma 2)."""
    rng = np.random.default_rng(1)
    for case in range(300):
        d = int(rng.integers(1, 4))
        L = int(rng.integers(0, 3 if d == 3 else 4))
        ncell = 1 << (L * d)
        occ = (rng.random(ncell) < rng.random()).astype(np.uint8)
        dom, key, cand, n = oracle.cell_classes(occ, d, L)
        assert n == cand_count(1 << L, d), (d, L)
        # candidate cells are never dominated, key cells are non-empty
        assert not (cand & dom).any()
        assert (occ[key.astype(bool)] == 1).all()


# ---- Theorem 1's bijection, written from Eqs. 9-15 (proof device) ----

def _keys_with_aux(key, d, L):
    G = 1 << L
    ks = [oracle.cell_columns(k, d, L) for k in np.flatnonzero(key)]
    for j in range(d):
        ks.append(tuple(G - 1 if k == j else -1 for k in range(d)))
    return ks


def _pdom(a, b):  # a partially dominates b (Def. 3), a assumed non-empty
    return all(x <= y for x, y in zip(a, b)) and any(x == y for x, y in zip(a, b))


def _Omega(c, key, d, L):
    Kc = [ck for ck in _keys_with_aux(key, d, L) if _pdom(ck, c)]
    omega = [max(j for j in range(d) if c[j] == ck[j]) for ck in Kc]  # Eq. 9
    return min(omega)                                                   # Eq. 10


def _Psi(c, key, d, L):  # Eq. 11
    G = 1 << L
    j = _Omega(c, key, d, L)
    return tuple(G - 1 if k == j else c[k] for k in range(d))


def _gamma(ca, G):  # Eq. 13
    return min(j for j in range(len(ca)) if ca[j] == G - 1)


def _Phi(ca, key, d, L):  # Eq. 14
    G = 1 << L
    g = _gamma(ca, G)
    vals = [ck[g] for ck in _keys_with_aux(key, d, L)
            if all(ck[j] <= ca[j] for j in range(g + 1))
            and all(ck[j] < ca[j] for j in range(g + 1, d))]
    return min(vals)


def _Theta(ca, key, d, L):  # Eq. 12
    G = 1 << L
    g = _gamma(ca, G)
    phi = _Phi(ca, key, d, L)
    return tuple(phi if k == g else ca[k] for k in range(d))


def test_theorem1_bijection_random():
    rng = np.random.default_rng(7)
    for case in range(120):
        d = int(rng.integers(2, 4))
        L = int(rng.integers(1, 3))
        G = 1 << L
        occ = (rng.random(1 << (L * d)) < rng.uniform(0.05, 0.5)).astype(np.uint8)
        dom, key, cand, n = oracle.cell_classes(occ, d, L)
        C = [oracle.cell_columns(k, d, L) for k in np.flatnonzero(cand)]
        CA = {c for c in (oracle.cell_columns(k, d, L) for k in range(1 << (L * d)))
              if any(x == G - 1 for x in c)}
        img = [_Psi(c, key, d, L) for c in C]
        assert len(set(img)) == len(C)          # injective
        assert set(img) == CA                   # onto CA_i (Lemma 2)
        for ca in CA:                           # Theta is the inverse
            assert _Psi(_Theta(ca, key, d, L), key, d, L) == ca


# ------------------------------------------------------ across layers ---

@pytest.mark.parametrize("kind", ["independent", "anticorrelated", "correlated"])
def test_corollaries_3_4_and_soundness(kind):
    d = 2 if kind != "independent" else 3
    P = skydata.generate(kind, 400, d, seed=21)
    S = oracle.skyline_brute(P)
    prev = None
    for L in range(0, 5 if d == 2 else 4):
        keys = oracle.cell_keys(P, L, assume_unit=True)
        occ = oracle.occupancy(keys, d, L)
        dom, key, cand, n = oracle.cell_classes(occ, d, L)
        assert n == cand_count(1 << L, d)
        # no skyline point lies in a dominated cell; each lies in a candidate cell
        assert not dom[keys[S].astype(np.int64)].any()
        assert cand[keys[S].astype(np.int64)].all()
        # every point of a dominated cell is dominated by a point (Def. 3 soundness)
        for i in np.flatnonzero(dom[keys.astype(np.int64)])[:50]:
            assert oracle.dominator(P, int(i)) >= 0
        if prev is not None:
            pkey, pcand, pL = prev
            kids = lambda c: [oracle.cell_key(tuple(2 * c[k] + ((b >> k) & 1) for k in range(d)), L)
                              for b in range(1 << d)]
            # Corollary 3: a key cell of layer L-1 splits into at least one key cell of layer L
            for k in np.flatnonzero(pkey):
                assert any(key[x] for x in kids(oracle.cell_columns(k, d, pL)))
            # Corollary 4: every key cell of layer L comes from a candidate cell of layer L-1
            for k in np.flatnonzero(key):
                parent = tuple(c // 2 for c in oracle.cell_columns(k, d, L))
                assert pcand[oracle.cell_key(parent, pL)]
        prev = (key, cand, L)


def test_dominated_cells_box_identity_matches_enumeration():
    """Two computations of Definition 3 agree: enumeration over all cell
    pairs (C) and the cumulative-OR box identity (numpy)."""
    rng = np.random.default_rng(21)
    for d, lg in [(1, 5), (2, 3), (2, 4), (3, 2), (3, 3), (4, 2), (5, 1), (6, 1)]:
        ncell = 1 << (lg * d)
        for density in (0.01, 0.1, 0.5):
            occ = (rng.random(ncell) < density).astype(np.uint8)
            dom, _, _, _ = oracle.cell_classes(occ, d, lg)
            assert np.array_equal(oracle.dominated_cells(occ, d, lg), dom), (d, lg, density)
    # one occupied cell dominates exactly the cells strictly above it
    d, lg = 3, 2
    occ = np.zeros(64, np.uint8)
    occ[oracle.cell_key((1, 0, 2), lg)] = 1
    dom = oracle.dominated_cells(occ, d, lg)
    want = [oracle.cell_key((a, b, c), lg) for a in range(2, 4) for b in range(1, 4) for c in range(3, 4)]
    assert sorted(np.flatnonzero(dom).tolist()) == sorted(want)
