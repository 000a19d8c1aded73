"""Parity of the refinement's paths with the oracle on inputs built to reach
them: the ring path, the sparse tail (a p-tile with at most a few live points
walking the remaining q-tiles itself), equal codes that need the exact float
test, exact duplicates (kept: neither dominates the other), and the long
Morton tie runs of correlated data. Exact equality of the index arrays."""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def gpu(P, **kw):
    x = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    return sky.skyline(x, **kw).cpu().numpy().tolist()


@pytest.mark.parametrize("d", [2, 3, 5, 8, 12, 16])
def test_duplicates_and_exact_ties(d):
    """Every point three times, coordinates on a coarse lattice (many equal
    codes and equal floats): duplicates of skyline points are all kept."""
    rng = np.random.default_rng(40 + d)
    base = (rng.integers(0, 24, size=(6000, d)) / 24.0).astype(np.float32)
    P = np.concatenate([base, base, base])[rng.permutation(18000)]
    want = oracle.skyline_sfs(P).tolist()
    assert gpu(P) == want
    assert gpu(P, assume_unit=True) == want


@pytest.mark.parametrize("kind,n,d", [("independent", 200000, 6), ("correlated", 200000, 8),
                                      ("anticorrelated", 60000, 5), ("independent", 120000, 12)])
def test_sparse_tail_sets(kind, n, d):
    """Sets whose p-tiles end with one or two live points (the sparse tail)
    and, for correlated data, long runs of equal Morton keys."""
    P = skydata.generate(kind, n, d, seed=7)
    want = oracle.skyline_sfs(P).tolist()
    assert gpu(P) == want
    st = sky.last_run_stats()
    assert st["skyline"] == len(want)


def test_few_points_far_apart_in_morton_order():
    """Skyline points spread over the whole Morton range, each the last live
    point of its tile, against many dominated points: every tile's tail runs
    the sparse walk to the end of its cutoff."""
    rng = np.random.default_rng(3)
    n, d = 150000, 4
    P = rng.random((n, d), dtype=np.float32) * 0.5 + 0.5          # dominated bulk in the upper half
    front = rng.random((64, d), dtype=np.float32)
    front /= front.sum(axis=1, keepdims=True)                     # an anti-chain near the origin
    front *= 0.45
    P[rng.choice(n, 64, replace=False)] = front
    want = oracle.skyline_sfs(P).tolist()
    assert gpu(P) == want


@pytest.mark.parametrize("d", [13, 16])
@pytest.mark.parametrize("kind", ["independent", "anticorrelated", "correlated"])
def test_high_dimension_ragged_tile_counts(kind, d):
    """Padded dimension 16 (13 and 16 dimensions): tile counts odd and even,
    a last tile with one point, sets spanning many CTAs of the refinement,
    with and without the sparse tail (the 256-point p-tile variant of the
    refinement, when built, meets the same cases: a last CTA with and
    without its second tile)."""
    for n in (129, 255, 256, 257, 385, 1000, 4097, 9001, 33000):
        P = skydata.generate(kind, n, d, seed=n + d)
        want = oracle.skyline_sfs(P).tolist()
        assert gpu(P) == want, (kind, d, n)
        assert gpu(P, assume_unit=True) == want, (kind, d, n)
