"""Writes fullsize_oracle.json: the oracle's skylines of the full-size workloads.

Run from the repository root:

    python tests/golden/make_fullsize.py [--only NAME[,NAME...]] [--threads T]

Every value in the output comes from ``oracle.skyline_sfs`` (the sort-first
skyline of Definitions 1-2) or ``oracle.skyline_subset`` on inputs drawn by
``skydata`` with the seeds the tests use; nothing here calls the CUDA library.
An index set is stored as its size and the SHA-256 of its ascending indices
as little-endian int32 (plus the first and last few indices, to help reading
a mismatch). The GPU parity tests compare the library's result with these.

Entries already in the file are kept, so an interrupted run resumes where it
stopped. The sets (names as in the file):

  c1            n = 2*10^4, d = 4, independent, seed 0
  c2-<kind>     n = 10^6, d = 8, seed 1, kind in independent / correlated /
                anticorrelated
  c3-independent n = 10^7, d = 12, independent, seed 1
  c5-rho<r>     n = 10^7, d = 8, Gaussian copula, rho in {0, 0.8}, seed 3
  c4            the 4,096 batched queries (seed 2) on the 20M x 12 mixed table
                (seed 2): one (size, hash) pair per query

Three workloads are not here because the sort-first oracle's cost grows
with the square of the skyline: the anti-correlated n = 10^7, d = 16 set
(8.2 * 10^6 skyline points), the copula set with rho = -0.8 (6.7 * 10^6) and
the batched queries with the largest skylines (up to ~10^6 each) would take
days on a few cores. Their tests check a dominating witness for every dropped
point instead, plus a sample of the kept points; for c4 the queries are
taken cheapest first and the file records how many were done.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import skydata  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_oracle.json")

C4_ROWS, C4_COLS, C4_QUERIES, C4_SEED = 20_000_000, 12, 4096, 2


def digest(idx) -> dict:
    a = np.ascontiguousarray(np.asarray(idx, dtype="<i4"))
    return {"count": int(a.size), "sha256": hashlib.sha256(a.tobytes()).hexdigest(),
            "first": a[:5].tolist(), "last": a[-5:].tolist()}


def sets():
    yield "c1", lambda: skydata.generate("independent", 20_000, 4, 0)
    for kind in ("independent", "correlated", "anticorrelated"):
        yield f"c2-{kind}", (lambda k=kind: skydata.generate(k, 1_000_000, 8, 1))
    yield "c3-independent", lambda: skydata.generate("independent", 10_000_000, 12, 1)
    for rho in (0.0, 0.8):
        yield f"c5-rho{rho:+.1f}", (lambda r=rho: skydata.copula(10_000_000, 8, 3, r)[0])


def load():
    if os.path.exists(OUT):
        with open(OUT) as f:
            return json.load(f)
    return {"written_by": "tests/golden/make_fullsize.py (oracle.skyline_sfs / oracle.skyline_subset only)",
            "hash": "sha256 of the ascending indices as little-endian int32",
            "sets": {}, "c4": None}


def save(doc):
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    os.replace(tmp, OUT)


def c4_cost_proxy(row_begin, row_count, dim_mask):
    """Rough relative cost of the oracle on one query, for the order only:
    the sort-first oracle's cost grows with the square of the skyline, which
    is small for independent rows (rows below C4_ROWS / 2) and a large share
    of the rows for anti-correlated ones (the upper half), more so at high d."""
    d = bin(dim_mask).count("1")
    half = C4_ROWS // 2
    anti = max(0, row_begin + row_count - max(row_begin, half)) / row_count
    sky = row_count * (anti * min(1.0, 0.08 * d * d / 12) + (1 - anti) * min(1.0, 0.002 * 2 ** d))
    return sky * sky + row_count * d


def run_c4(doc, threads, budget):
    T = skydata.mixed_table(C4_ROWS, C4_COLS, C4_SEED)
    Q = skydata.batched_queries(C4_QUERIES, C4_ROWS, C4_COLS, C4_SEED)
    c4 = doc.get("c4") or {"table": f"skydata.mixed_table({C4_ROWS}, {C4_COLS}, seed={C4_SEED})",
                           "queries": f"skydata.batched_queries({C4_QUERIES}, {C4_ROWS}, {C4_COLS}, seed={C4_SEED})",
                           "per_query": [None] * C4_QUERIES, "oracle_seconds": 0.0}
    doc["c4"] = c4
    # cheapest queries first, so that a run stopped by its time budget has
    # covered as many queries as possible
    order = sorted(range(C4_QUERIES), key=lambda i: c4_cost_proxy(*(int(v) for v in Q[i])))
    last = start = time.time()
    for i in order:
        if c4["per_query"][i] is not None:
            continue
        if budget and time.time() - start > budget:
            break
        r0, cnt, mask = (int(v) for v in Q[i])
        t0 = time.perf_counter()
        S = oracle.skyline_subset(T, r0, cnt, mask, threads=threads)
        c4["oracle_seconds"] += time.perf_counter() - t0
        dg = digest(S)
        c4["per_query"][i] = [dg["count"], dg["sha256"][:16]]
        if time.time() - last > 60:
            save(doc)
            last = time.time()
            done = sum(v is not None for v in c4["per_query"])
            print(f"c4: {done}/{C4_QUERIES} queries, oracle {c4['oracle_seconds']:.0f} s", flush=True)
    c4["queries_done"] = sum(v is not None for v in c4["per_query"])
    save(doc)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="", help="comma-separated names (c1, c2-independent, ..., c4)")
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: all cores)")
    ap.add_argument("--budget-seconds", type=float, default=0.0,
                    help="c4: take no new query after this many seconds (0: no limit)")
    args = ap.parse_args()
    only = {s for s in args.only.split(",") if s}
    doc = load()
    for name, make in sets():
        if (only and name not in only) or name in doc["sets"]:
            continue
        P = make()
        t0 = time.perf_counter()
        S = oracle.skyline_sfs(P, args.threads)
        sec = time.perf_counter() - t0
        doc["sets"][name] = {"n": int(P.shape[0]), "d": int(P.shape[1]), **digest(S),
                             "oracle_seconds": round(sec, 1), "threads": args.threads or oracle.max_threads()}
        save(doc)
        print(f"{name}: |S| = {S.size}, {sec:.1f} s", flush=True)
    if not only or "c4" in only:
        run_c4(doc, args.threads, args.budget_seconds)


if __name__ == "__main__":
    main()
