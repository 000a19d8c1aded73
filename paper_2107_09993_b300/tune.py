"""Autotuner for the batched skyline path (sky_batch_create's tuning knobs).

The batched launch runs steps (a)-(c) for every query and then one persistent
refinement kernel per padded-dimension class (class c: queries of 4c+1 ..
4c+4 attributes). The knobs below change the time of a batch, never its
result:

* per (d, log2 n) bucket: the grid layer of its queries (2^log2_g cells per
  dimension; finer grids prune more in step (c) but cost more bitmap work),
  as an offset from the automatic layer;
* per class, the shape and split of the refinement:
  - the ring depth of streamed q-tiles in shared memory (4 or 8 stages of
    128 points),
  - the pair test of the list probe (7-bit codes, or 3-bit fast codes first),
  - persistent CTAs per SM (the work split of the (query, p-tile) items);
  the classes of 9-16 attributes test pairs by threshold masks with a fixed
  4-stage ring (the library's mask probe), so for them only the CTAs per SM
  remain a knob;
* whether the class kernels run one after another or as parallel branches
  of the graph (their tails overlap).

`tune()` times candidates on a sample of the caller's own queries by
coordinate descent (layers per bucket, then each class's variant on that
class's queries, then class concurrency), compares the result with the
library defaults on the whole sample, keeps the defaults unless the tuned
choice is faster, and stores it in a JSON cache keyed by GPU name.
`settings()` turns the cache into the knobs `Batch` accepts; `Batch` applies
the cache by default.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning.json")
MAX_GRID_BITS = 18  # batched grids hold at most 2^18 cells
MAX_AUTO_LAYER = 8  # the automatic layer never exceeds 8 (256 columns per dimension)
CTAS = (0, 2, 4)     # persistent CTAs per SM candidates (0: as many as fit)
STAGES = (8, 4)
CODES = (1, 2)       # 1: 7-bit codes, 2: 3-bit fast codes first
MASK_CLASSES = (2, 3)  # classes whose refinement uses the mask probe (depth and pair test fixed)


def auto_log2g(n: int, d: int) -> int:
    """The library's automatic layer for a batched query (mirrors the C++ rule)."""
    r = max(1, min(MAX_AUTO_LAYER, 24 // d))
    while r > 1 and (1 << (r * d)) > 32.0 * max(n, 1):
        r -= 1
    while r > 1 and r * d > MAX_GRID_BITS:
        r -= 1
    return r


def bucket(n: int, d: int) -> str:
    return f"d{d}_n{int(math.log2(max(n, 1)))}"


def _dims(mask: int) -> int:
    return bin(int(mask) & 0xffffffff).count("1")


def _class(d: int) -> int:
    return (d - 1) // 4


def default_knobs() -> dict:
    """The library's defaults, as knobs (3-bit fast codes in class 3 only)."""
    return {"class_ctas": [0, 0, 0, 0], "class_stages": [8, 8, 8, 8], "class_code": [1, 1, 1, 2],
            "concurrent_classes": 0, "layer_offset": {}}


def layers_for(queries, offsets: dict) -> np.ndarray:
    q = np.asarray(queries, dtype=np.int64).reshape(-1, 3)
    out = []
    for _, n, m in q:
        d = _dims(m)
        if d < 1 or d > 16 or int(m) >> 32:
            out.append(-1)   # automatic: the library checks the query and reports it
            continue
        lg = auto_log2g(int(n), d) + int(offsets.get(bucket(int(n), d), 0))
        lg = max(0, lg)
        while lg > 0 and lg * d > MAX_GRID_BITS:
            lg -= 1
        out.append(lg)
    return np.array(out, dtype=np.int32)


def _knobs_for(queries, k: dict) -> dict:
    return {"class_ctas": k["class_ctas"], "class_stages": k["class_stages"], "class_code": k["class_code"],
            "concurrent_classes": k["concurrent_classes"], "log2g": layers_for(queries, k["layer_offset"])}


def _time(sky, table, queries, knobs, repeats):
    """Median device time (ms) of `repeats` launches of one bound batch."""
    import torch
    b = sky.Batch(table, queries, tuning=_knobs_for(queries, knobs))
    b.run()
    ms = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    b.close()
    return statistics.median(ms)


def tune(table, queries, sample: int = 512, per_bucket: int = 8, repeats: int = 3,
         cache_path: str | None = DEFAULT_CACHE, seed: int = 0, verbose: bool = False) -> dict:
    """Tunes the knobs on a sample of `queries` (int array [n, 3]: row_begin,
    row_count, dim_mask) over `table` (the CUDA tensor Batch takes). Returns
    the cache entry: the chosen knobs, the sample's time with the library
    defaults and with the chosen knobs (ms), and what was tried."""
    import torch
    import paper_2107_09993_b300 as sky

    t_start = time.time()
    rng = np.random.default_rng(seed)
    q = np.asarray(queries, dtype=np.int64).reshape(-1, 3)
    pick = np.sort(rng.choice(len(q), size=min(len(q), sample), replace=False))
    S = q[pick]
    best = default_knobs()
    tried = []

    def timed(qs, k, what):
        ms = _time(sky, table, qs, k, repeats)
        tried.append({"what": what, "queries": int(len(qs)), "ms": round(ms, 3)})
        if verbose:
            print(f"[tune] {what}: {ms:.3f} ms ({len(qs)} queries)", flush=True)
        return ms

    # 1. grid layer per (d, log2 n) bucket, on up to per_bucket of its queries
    groups: dict[str, list[int]] = {}
    for i, (_, n, m) in enumerate(S):
        groups.setdefault(bucket(int(n), _dims(m)), []).append(i)
    for key, idx in sorted(groups.items()):
        sel = S[rng.choice(idx, size=min(per_bucket, len(idx)), replace=False)]
        d = _dims(sel[0, 2])
        base = auto_log2g(int(np.median(sel[:, 1])), d)
        res = []
        for off in (0, -1, 1):
            lg = base + off
            if lg < 0 or lg * d > MAX_GRID_BITS:
                continue
            k = dict(best, layer_offset={key: off})
            res.append((timed(sel, k, f"layer {key} {off:+d}"), off))
        best["layer_offset"][key] = min(res)[1]
    # 2. each class's refinement variant, on that class's queries
    for c in range(4):
        sel = S[[_class(_dims(m)) == c for _, _, m in S]]
        if len(sel) == 0:
            continue
        res = []
        fixed = c in MASK_CLASSES
        for code in ((best["class_code"][c],) if fixed else CODES):
            for st in ((best["class_stages"][c],) if fixed else STAGES):
                for ctas in CTAS:
                    k = json.loads(json.dumps(best))
                    k["class_code"][c], k["class_stages"][c], k["class_ctas"][c] = code, st, ctas
                    ms = timed(sel, k, f"class {c}: code {code} stages {st} ctas {ctas}")
                    res.append((ms, code, st, ctas))
        _, best["class_code"][c], best["class_stages"][c], best["class_ctas"][c] = min(res)
    # 3. class kernels one after another or concurrently, on the whole sample
    res = []
    for conc in (0, 1):
        k = dict(best, concurrent_classes=conc)
        res.append((timed(S, k, f"concurrent classes {conc}"), conc))
    best["concurrent_classes"] = min(res)[1]
    # 4. the chosen knobs against the library defaults, interleaved
    t_def, t_tuned = [], []
    for _ in range(3):
        t_def.append(timed(S, default_knobs(), "defaults"))
        t_tuned.append(timed(S, best, "tuned"))
    md, mt = statistics.median(t_def), statistics.median(t_tuned)
    if mt > md:   # the defaults were not beaten: keep them
        best, mt = default_knobs(), md
    entry = dict(best, default_ms=round(md, 3), tuned_ms=round(mt, 3), sample_queries=int(len(S)),
                 tuned_s=round(time.time() - t_start, 1), candidates=len(tried))
    if cache_path:
        gpu = torch.cuda.get_device_name()
        cache = load_cache(cache_path)
        cache[gpu] = entry
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
            f.write("\n")
    entry["tried"] = tried
    return entry


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def settings(queries, cache: dict | None = None, gpu: str | None = None) -> dict | None:
    """Knobs for `Batch(tuning=...)` from a tuning cache: per-query layers
    (automatic layer + the bucket's offset) and the class variants; None
    when the cache has no entry for this GPU."""
    if cache is None:
        cache = load_cache()
    if not cache:
        return None
    if gpu is None:
        import torch
        gpu = torch.cuda.get_device_name()
    entry = cache.get(gpu)
    if not entry:
        return None
    k = default_knobs()
    for key in ("class_ctas", "class_stages", "class_code", "concurrent_classes", "layer_offset"):
        if key in entry:
            k[key] = entry[key]
    return _knobs_for(queries, k)
