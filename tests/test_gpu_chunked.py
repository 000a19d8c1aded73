"""sky_skyline_chunked (sets beyond one in-core call) against the oracle and
against the in-core path: device and host input, ragged chunk sizes, every
value-map mode, the candidates of step (c), and the error paths."""
import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("kind,n,d,chunk", [("independent", 60000, 4, 7001), ("anticorrelated", 20000, 3, 4096),
                                            ("correlated", 90000, 6, 33333), ("independent", 5000, 9, 100),
                                            ("anticorrelated", 12345, 2, 12345), ("independent", 40000, 1, 999)])
def test_chunked_matches_oracle_device_and_host(kind, n, d, chunk):
    P = skydata.generate(kind, n, d, seed=n % 97)
    want = oracle.skyline_sfs(P).tolist()
    got = sky.skyline_chunked(dev(P), chunk_rows=chunk).cpu().tolist()
    assert got == want
    host = torch.from_numpy(P).pin_memory()
    assert sky.skyline_chunked(host, chunk_rows=chunk).cpu().tolist() == want
    assert sky.skyline_chunked(P, chunk_rows=chunk).cpu().tolist() == want          # pageable numpy


def test_chunked_equals_in_core_path_and_modes():
    for i, (kind, n, d) in enumerate([("independent", 300000, 8), ("correlated", 250000, 5),
                                      ("anticorrelated", 200000, 6)]):
        P = skydata.generate(kind, n, d, seed=60 + i)
        if i == 1:
            P = (P * np.float32(0.2) + np.float32(0.3)).astype(np.float32)      # automatic map normalises
        x = dev(P)
        for mode in (0, 1, 2):
            want = sky.skyline(x, assume_unit=mode).long()
            got = sky.skyline_chunked(x, assume_unit=mode, chunk_rows=65536 + 17 * i)
            assert torch.equal(got, want), (kind, mode)
            # step (c) alone: the same candidates as the in-core call
            c_in = sky.skyline(x, assume_unit=mode, survivors_only=True).long()
            c_ch = sky.skyline_chunked(x, assume_unit=mode, survivors_only=True, chunk_rows=40000)
            assert torch.equal(c_ch, c_in), (kind, mode)


def test_chunked_strided_host_rows():
    P = skydata.generate("independent", 30000, 7, seed=3)
    wide = np.zeros((30000, 10), np.float32)
    wide[:, :7] = P
    view = torch.from_numpy(wide)[:, :7]                # row stride 10 floats
    assert sky.skyline_chunked(view, chunk_rows=4000).cpu().tolist() == oracle.skyline_sfs(P).tolist()
    assert sky.skyline_chunked(view.cuda(), chunk_rows=4000).cpu().tolist() == oracle.skyline_sfs(P).tolist()


def test_chunked_errors():
    P = skydata.generate("anticorrelated", 20000, 4, seed=5)
    x = dev(P)
    want = oracle.skyline_sfs(P)
    with pytest.raises(sky.SkyError) as e:
        sky.skyline_chunked(x, chunk_rows=3000, capacity=len(want) - 1)
    assert e.value.name == "SKY_ERR_CAPACITY" and f"count={len(want)}" in str(e.value)
    with pytest.raises(sky.SkyError) as e:
        sky.skyline_chunked(x, chunk_rows=3000, max_candidates=100)
    assert e.value.name == "SKY_ERR_CAPACITY" and "candidates" in str(e.value)
    bad = P.copy()
    bad[17000, 2] = np.inf
    with pytest.raises(sky.SkyError) as e:
        sky.skyline_chunked(dev(bad), chunk_rows=3000)
    assert e.value.name == "SKY_ERR_NONFINITE"
    assert sky.skyline_chunked(torch.empty((0, 3), dtype=torch.float32, device="cuda")).numel() == 0
