"""The tournament-tree ShrinkKeyCells (Algorithm 3, as read in the library:
all cells are leaves, one dimension per pass) against the oracle.

Theorem 2: the tree's pointers give the key cells (l(c) = c), the
candidate cells and, through the cell one step down the diagonal, the
dominated cells -- the same sets as Definitions 3-6 enumerate
(oracle.cell_classes) and as the prefix-OR path computes (Grid)."""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def _words(occ):
    occ = np.asarray(occ, dtype=np.uint8)
    n = occ.size
    w = np.zeros(max(1, (n + 31) // 32), dtype=np.uint32)
    idx = np.flatnonzero(occ)
    np.bitwise_or.at(w, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return torch.from_numpy(w.view(np.int32)).cuda()


def _classes(occ, d, lg):
    cls = sky.tournament_cells(_words(occ), d, lg).cpu().numpy()
    return (cls & 1).astype(np.uint8), ((cls >> 1) & 1).astype(np.uint8), ((cls >> 2) & 1).astype(np.uint8)


def test_random_layers_match_the_oracle():
    rng = np.random.default_rng(31)
    for case in range(60):
        d = int(rng.integers(1, 5))
        lg = int(rng.integers(0, {1: 8, 2: 5, 3: 3, 4: 3}[d]))
        ncell = 1 << (lg * d)
        density = [0.02, 0.1, 0.3, 0.7][case % 4]
        occ = (rng.random(ncell) < density).astype(np.uint8)
        dom, key, cand, _ = oracle.cell_classes(occ, d, lg)
        got = _classes(occ, d, lg)
        assert np.array_equal(got[0], dom), (case, d, lg, "dominated")
        assert np.array_equal(got[1], key), (case, d, lg, "key")
        assert np.array_equal(got[2], cand), (case, d, lg, "candidate")


def test_fig1_layer4_key_cells(golden):
    """The Fig. 1 reconstruction (Layer 4 of a 2-d data set): the key cells
    and the 31 candidate cells the paper states."""
    g = golden("fig1_layer4.json")
    lg, d = g["log2g"], g["d"]
    key_cells = [(c0, c1) for c1, c0 in g["key_cells_c1_c0"]]
    occ = np.zeros(1 << (lg * d), dtype=np.uint8)
    for c in key_cells:
        occ[oracle.cell_key(c, lg)] = 1
    dom, key, cand = _classes(occ, d, lg)
    assert sorted(np.flatnonzero(key).tolist()) == sorted(oracle.cell_key(c, lg) for c in key_cells)
    assert int(cand.sum()) == g["n_candidates"]
    want_dom, want_key, want_cand, _ = oracle.cell_classes(occ, d, lg)
    assert np.array_equal(key, want_key) and np.array_equal(cand, want_cand) and np.array_equal(dom, want_dom)


def test_point_sets_match_the_prefix_or_path():
    """On the occupancy of real point sets (up to 2^20 cells), the
    tournament's dominated cells equal the prefix-OR path's (Grid), and its
    key and candidate cells equal the oracle's box-identity counterparts."""
    for kind, n, d, lg in (("independent", 200_000, 4, 5), ("anticorrelated", 100_000, 5, 4),
                           ("correlated", 50_000, 10, 2), ("anticorrelated", 30_000, 16, 1)):
        P = skydata.generate(kind, n, d, seed=d)
        g = sky.Grid(torch.from_numpy(P).cuda(), log2_g=lg, assume_unit=True).prune()
        words = g.occupied()
        dom, key, cand = (x for x in _classes_from_words(words, d, lg))
        want_dom = _bits(g.dominated(), 1 << (lg * d))
        assert np.array_equal(dom, want_dom), (kind, n, d)
        occ = _bits(words, 1 << (lg * d))
        box = oracle.dominated_cells(occ, d, lg)
        assert np.array_equal(dom, box)
        # key cell: occupied, and no other occupied cell <= it
        assert np.array_equal(key, _keys_by_box(occ, d, lg)), (kind, n, d)
        assert cand.sum() >= key.sum()
        g.close()


def _classes_from_words(words, d, lg):
    cls = sky.tournament_cells(words, d, lg).cpu().numpy()
    return (cls & 1).astype(np.uint8), ((cls >> 1) & 1).astype(np.uint8), ((cls >> 2) & 1).astype(np.uint8)


def _bits(words, n):
    w = words.cpu().numpy().view(np.uint32)
    return ((w[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1).astype(np.uint8)


def _keys_by_box(occ, d, lg):
    """Key cells through the oracle's box identity: c is a key cell iff it is
    occupied and none of the boxes [0, c - e_k] holds an occupied cell."""
    G = 1 << lg
    occb = np.asarray(occ, dtype=bool).reshape((G,) * d)
    box = occb
    for ax in range(d):
        box = np.logical_or.accumulate(box, axis=ax)
    other = np.zeros_like(occb)
    for ax in range(d):
        sl_dst = [slice(None)] * d
        sl_src = [slice(None)] * d
        sl_dst[ax] = slice(1, None)
        sl_src[ax] = slice(0, -1)
        other[tuple(sl_dst)] |= box[tuple(sl_src)]
    return (occb & ~other).astype(np.uint8).reshape(-1)


def test_limits():
    assert sky.load().sky_tournament_workspace_size(16, 2) == 0     # 2^32 cells
    with pytest.raises(sky.SkyError):
        sky.tournament_cells(torch.zeros(4, dtype=torch.int32, device="cuda"), 14, 2)
