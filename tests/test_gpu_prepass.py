"""The refinement's pre-pass (sets of at least 2^21 rows): every p-tile first
meets its own tile and the first Morton tiles, the survivors are compacted
and the full refinement runs on them. These sets sit just above the row
threshold with ragged sizes; their skylines are small enough for the
oracle's whole result, so the check is exact equality (Definitions 1-2).
Also: witness mode names a dominator for every row the pre-pass removes, and
a set whose step (c) leaves fewer than 2^21 survivors (the device skips the
pre-pass, the compaction keeps every entry) gives the same exact result."""
import numpy as np
import pytest

import oracle
import skydata
from parity import check_witnesses

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402

N_PRE = 1 << 21


@pytest.mark.parametrize("kind,n,d,seed", [
    ("independent", 2_200_001, 5, 11),      # the pre-pass removes most survivors
    ("independent", 2_300_003, 4, 12),
    ("anticorrelated", 2_700_017, 3, 13),
])
def test_prepass_sets_equal_oracle(kind, n, d, seed):
    """Layer 1 (two columns per dimension): step (c) can drop only the
    all-ones cell, so at least 2^21 survivors reach the refinement and its
    pre-pass runs."""
    P = skydata.generate(kind, n, d, seed)
    want = oracle.skyline_sfs(P)
    x = torch.from_numpy(P).cuda()
    got = sky.skyline(x, log2_g=1).cpu().numpy()
    st = sky.last_run_stats()
    assert st["survivors"] >= N_PRE, "the pre-pass must be active for this case"
    assert np.array_equal(got, want)
    S, W = sky.skyline_witness(x, log2_g=1)
    assert np.array_equal(S.cpu().numpy(), want)
    check_witnesses(P, want, W.cpu().numpy())


def test_prepass_skipped_below_the_survivor_threshold():
    """Correlated rows: step (c) leaves far fewer than 2^21 survivors, so the
    pre-pass kernel returns at once and the compaction keeps every entry."""
    P = skydata.generate("correlated", N_PRE + 4_321, 6, 14)
    want = oracle.skyline_sfs(P)
    x = torch.from_numpy(P).cuda()
    got = sky.skyline(x).cpu().numpy()
    assert sky.last_run_stats()["survivors"] < N_PRE
    assert np.array_equal(got, want)
    assert np.array_equal(sky.skyline(x).cpu().numpy(), want)   # the cached graph


def test_prepass_times_out_then_recovers():
    """With the pipeline's poll limit at 1, a call through the pre-pass (its
    compaction's look-back included) reports SKY_ERR_TIMEOUT and stays inside
    its arrays; with the default limit the next call is exact again."""
    P = skydata.generate("independent", 2_200_001, 5, 11)
    want = oracle.skyline_sfs(P)
    x = torch.from_numpy(P).cuda()
    timed_out = False
    sky.set_wait_limit(1)
    try:
        for _ in range(3):
            try:
                sky.skyline(x, log2_g=1)
            except sky.SkyError as e:
                assert e.status == 7, e   # SKY_ERR_TIMEOUT
                timed_out = True
                break
    finally:
        sky.set_wait_limit(0)
    assert timed_out
    assert np.array_equal(sky.skyline(x, log2_g=1).cpu().numpy(), want)
