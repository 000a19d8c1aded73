"""The stored full-size oracle results (tests/golden/fullsize_oracle.json) are
the oracle's: the entries that the oracle recomputes in seconds are recomputed
here on the CPU and compared with the file (size, SHA-256, first and last
indices), and every entry is checked for the fields the GPU parity tests read.
No GPU, no CUDA library."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import skydata

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_oracle.json")


def _doc():
    with open(GOLDEN) as f:
        return json.load(f)


def _digest(S):
    a = np.ascontiguousarray(np.asarray(S, dtype="<i4"))
    return a.size, hashlib.sha256(a.tobytes()).hexdigest(), a[:5].tolist(), a[-5:].tolist()


def test_golden_file_has_every_set():
    doc = _doc()
    sets = doc["sets"]
    for name in ("c1", "c2-independent", "c2-correlated", "c2-anticorrelated", "c3-independent",
                 "c5-rho+0.0", "c5-rho+0.8"):
        assert name in sets, name
        e = sets[name]
        assert e["count"] > 0 and len(e["sha256"]) == 64
        assert len(e["first"]) == min(5, e["count"])
    c4 = doc["c4"]
    assert c4 is not None and len(c4["per_query"]) == 4096
    done = [v for v in c4["per_query"] if v is not None]
    assert len(done) == c4["queries_done"] > 0
    assert all(isinstance(v[0], int) and len(v[1]) == 16 for v in done)


@pytest.mark.parametrize("name,kind,n,d,seed", [
    ("c1", "independent", 20_000, 4, 0),
    ("c2-correlated", "correlated", 1_000_000, 8, 1),
])
def test_cheap_entries_recomputed(name, kind, n, d, seed):
    e = _doc()["sets"][name]
    P = skydata.generate(kind, n, d, seed)
    S = oracle.skyline_sfs(P)
    cnt, sha, first, last = _digest(S)
    assert (e["n"], e["d"]) == (n, d)
    assert cnt == e["count"] and sha == e["sha256"]
    assert first == e["first"] and last == e["last"]


def test_c4_cheapest_query_recomputed():
    """One batched query's stored (size, hash prefix) equals the oracle's
    skyline of that query's rows and columns, recomputed here."""
    doc = _doc()["c4"]
    Q = skydata.batched_queries(4096, 20_000_000, 12, seed=2)
    # the smallest query that the file holds
    done = [i for i, v in enumerate(doc["per_query"]) if v is not None]
    i = min(done, key=lambda j: int(Q[j][1]) * bin(int(Q[j][2])).count("1"))
    r0, cnt, mask = (int(v) for v in Q[i])
    T = skydata.mixed_table(20_000_000, 12, seed=2)
    S = oracle.skyline_subset(T, r0, cnt, mask)
    size, sha, _, _ = _digest(S)
    assert [size, sha[:16]] == doc["per_query"][i]
