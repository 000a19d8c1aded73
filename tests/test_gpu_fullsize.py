"""Parity at the full workload sizes, in the launch configuration bench.py
times (default options, device-resident inputs, several sets per call).

Two kinds of evidence, both complete for what they cover:
* the oracle's whole result: the size and SHA-256 of the oracle's sorted
  index set (tests/golden/fullsize_oracle.json, written by
  tests/golden/make_fullsize.py from oracle.skyline_sfs) must equal those of
  the library's result;
* witnesses: the library's witness mode names, for every row it drops, a row
  that dominates it (Definition 1), checked here row by row. That proves every
  dropped row dominated, hence every skyline row returned.
Where the oracle cannot finish (its cost grows with the square of the skyline:
the anti-correlated n = 10^7, d = 16 set has 8.2 * 10^6 skyline points, the
rho = -0.8 copula set 6.7 * 10^6), the returned rows are checked on a sample
with the oracle's single-point test, on top of the witnesses."""
import numpy as np
import pytest

import skydata
from parity import check_kept_sample, check_witnesses, digest, golden_fullsize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def _golden(name):
    g = golden_fullsize()["sets"]
    assert name in g, f"{name} missing from the oracle file (run tests/golden/make_fullsize.py)"
    return g[name]


def _assert_oracle(S, name):
    g = _golden(name)
    assert S.size == g["count"], (name, S.size, g["count"])
    assert digest(S) == g["sha256"], (name, S[:5].tolist(), g["first"])


def test_config0_oracle_hash_pin():
    """The stored hash of the 2*10^4 x 4 set equals the oracle's result
    computed here (pins the hashing and the golden file itself)."""
    import oracle
    P = skydata.generate("independent", 20_000, 4, 0)
    S = oracle.skyline_sfs(P)
    _assert_oracle(S, "c1")
    got = sky.skyline(torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.array_equal(got, S)


def test_config1_three_sets_exact():
    """n = 10^6, d = 8, seed 1: the three sets in one sky_skyline_sets call
    (the bench's former step), each equal to the oracle's whole result, and
    every dropped row witnessed."""
    kinds = ("independent", "correlated", "anticorrelated")
    host = [skydata.generate(k, 1_000_000, 8, 1) for k in kinds]
    xs = [torch.from_numpy(P).cuda() for P in host]
    got = [r.cpu().numpy() for r in sky.skyline_sets(xs)]
    for k, P, x, S in zip(kinds, host, xs, got):
        _assert_oracle(S, f"c2-{k}")
        Sw, W = sky.skyline_witness(x)
        assert np.array_equal(Sw.cpu().numpy(), S)
        check_witnesses(P, S, W.cpu().numpy())
    # host-buffer entry point, same result
    S2 = sky.skyline_host(torch.from_numpy(host[2]).pin_memory()).numpy()
    assert np.array_equal(S2, got[2])


def test_config2_large_sets():
    """n = 10^7: anti-correlated d = 16 and independent d = 12, seed 1, in one
    sky_skyline_sets call (the bench's step). Independent: the oracle's whole
    result. Both: every dropped row witnessed; anti-correlated: 20,000
    returned rows checked with the oracle's single-point test."""
    specs = (("anticorrelated", 16), ("independent", 12))
    host = [skydata.generate(k, 10_000_000, d, 1) for k, d in specs]
    xs = [torch.from_numpy(P).cuda() for P in host]
    got = [r.cpu().numpy() for r in sky.skyline_sets(xs)]
    _assert_oracle(got[1], "c3-independent")
    for (kind, d), P, x, S in zip(specs, host, xs, got):
        Sw, W = sky.skyline_witness(x)
        assert np.array_equal(Sw.cpu().numpy(), S), kind
        check_witnesses(P, S, W.cpu().numpy())
        del W, Sw
    check_kept_sample(host[0], got[0], 20_000, 12)


@pytest.mark.parametrize("rho", [-0.8, 0.0, 0.8])
def test_config4_copula_eval_sets(rho):
    """The learned proposal's evaluation sets (n = 10^7, d = 8, seed 3), plain
    path: the oracle's whole result for rho = 0 and 0.8; witnesses for every
    dropped row and 20,000 sampled returned rows for rho = -0.8."""
    P, _ = skydata.copula(10_000_000, 8, 3, rho)
    x = torch.from_numpy(P).cuda()
    S = sky.skyline(x).cpu().numpy()
    if rho != -0.8:
        _assert_oracle(S, f"c5-rho{rho:+.1f}")
    Sw, W = sky.skyline_witness(x)
    assert np.array_equal(Sw.cpu().numpy(), S)
    check_witnesses(P, S, W.cpu().numpy())
    if rho == -0.8:
        check_kept_sample(P, S, 20_000, 13)
