"""Checks shared by the GPU parity tests (host side, no CUDA).

`check_witnesses` verifies the library's witness mode against Definition 1
directly: every row outside the returned skyline must carry the row of a point
that dominates it, and every returned row must carry -1. Together with a
check of the kept rows (the oracle's full result, or its single-point test
on a sample) this proves the returned set equal to the skyline: if every
dropped point is dominated, every undominated point was kept.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_oracle.json")


def golden_fullsize():
    with open(GOLDEN) as f:
        return json.load(f)


def digest(idx) -> str:
    a = np.ascontiguousarray(np.asarray(idx, dtype="<i4"))
    return hashlib.sha256(a.tobytes()).hexdigest()


def check_witnesses(P, S, W, chunk=1 << 21):
    """P: [n, d] float32 (host), S: ascending returned rows, W: [n] witnesses."""
    P = np.ascontiguousarray(P, dtype=np.float32)
    S = np.asarray(S, dtype=np.int64)
    W = np.asarray(W, dtype=np.int64)
    n = P.shape[0]
    assert W.shape == (n,)
    assert np.all(np.diff(S) > 0), "returned rows not strictly ascending"
    kept = np.zeros(n, dtype=bool)
    kept[S] = True
    bad_kept = np.flatnonzero(kept & (W != -1))
    assert bad_kept.size == 0, f"{bad_kept.size} returned rows carry a witness, e.g. {bad_kept[:5]}"
    drop = np.flatnonzero(~kept)
    w = W[drop]
    missing = drop[w < 0]
    assert missing.size == 0, (f"{missing.size} dropped rows without a witness "
                               f"(codes {np.unique(W[missing])[:3]}), e.g. {missing[:5]}")
    assert np.all(w < n)
    for s in range(0, drop.size, chunk):
        p = P[drop[s:s + chunk]]
        q = P[w[s:s + chunk]]
        ok = np.all(q <= p, axis=1) & np.any(q < p, axis=1)   # Definition 1: q dominates p
        assert ok.all(), f"witness does not dominate rows {drop[s:s + chunk][~ok][:5]}"
    return drop.size


def check_kept_sample(P, S, k, seed):
    """The oracle's single-point test on k sampled returned rows: none may
    have a dominator anywhere in P."""
    S = np.asarray(S)
    if S.size == 0:
        return 0
    rng = np.random.default_rng(seed)
    sample = rng.choice(S, size=min(k, S.size), replace=False)
    w = oracle.dominators(P, sample)
    assert np.all(w == -1), f"returned rows with a dominator: {sample[w != -1][:5]}"
    return sample.size
