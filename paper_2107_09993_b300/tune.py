"""Autotuner for the batched skyline path.

Two knobs decide the speed of a batch (never its result):

* the grid layer of each query (2^log2_g cells per dimension): finer grids
  prune more points in step (c) but cost more bitmap work;
* the work split of the persistent refinement (CTAs per SM pulling
  (query, tile) items).

`tune()` times candidate settings on sample batches drawn from the caller's
own queries, bucketed by (dimensions, log2 of row count), and keeps the
fastest per bucket; `settings()` turns a cache into the per-query layer array
and the CTAs-per-SM value that `Batch` accepts. The cache is a JSON file keyed
by GPU name.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning.json")
MAX_GRID_BITS = 18  # batched grids hold at most 2^18 cells
MAX_AUTO_LAYER = 8  # the automatic layer never exceeds 8 (256 columns per dimension)


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


def _time_batch(sky, table, queries, log2g, ctas, repeats):
    import torch
    b = sky.Batch(table, queries, log2g=log2g, refine_ctas_per_sm=ctas)
    best = float("inf")
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    b.close()
    return best


def tune(table, queries, per_bucket: int = 8, repeats: int = 3, cache_path: str = DEFAULT_CACHE,
         seed: int = 0, verbose: bool = False) -> dict:
    """Times layer offsets per bucket and the refinement split on samples of
    `queries` (int array [n, 3]: row_begin, row_count, dim_mask)."""
    import torch
    import paper_2107_09993_b300 as sky

    rng = np.random.default_rng(seed)
    q = np.asarray(queries, dtype=np.int64).reshape(-1, 3)
    groups: dict[str, list[int]] = {}
    for i, (_, n, m) in enumerate(q):
        groups.setdefault(bucket(int(n), _dims(m)), []).append(i)
    layers = {}
    t0 = time.time()
    for key, idx in sorted(groups.items()):
        pick = rng.choice(idx, size=min(per_bucket, len(idx)), replace=False)
        sample = q[pick]
        d = _dims(sample[0, 2])
        n = int(np.median(sample[:, 1]))
        base = auto_log2g(n, d)
        best = None
        for off in (-1, 0, 1):
            lg = base + off
            if lg < 0 or lg * d > MAX_GRID_BITS:
                continue
            ms = _time_batch(sky, table, sample, [lg] * len(sample), 0, repeats)
            if best is None or ms < best[1]:
                best = (off, ms)
        layers[key] = best[0]
        if verbose:
            print(f"[tune] {key}: layer offset {best[0]:+d} ({best[1]:.3f} ms)", flush=True)
    # refinement work split on a mixed sample
    pick = rng.choice(len(q), size=min(len(q), 256), replace=False)
    sample = q[pick]
    lgs = [auto_log2g(int(n), _dims(m)) + layers.get(bucket(int(n), _dims(m)), 0) for _, n, m in sample]
    split = None
    for ctas in (0, 1, 2, 3, 4):
        ms = _time_batch(sky, table, sample, lgs, ctas, repeats)
        if split is None or ms < split[1]:
            split = (ctas, ms)
        if verbose:
            print(f"[tune] refine CTAs/SM {ctas}: {ms:.3f} ms", flush=True)
    gpu = torch.cuda.get_device_name()
    cache = load_cache(cache_path)
    cache[gpu] = {"layer_offset": layers, "refine_ctas_per_sm": split[0],
                  "tuned_s": round(time.time() - t0, 1), "queries_sampled": int(len(q))}
    with open(cache_path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return cache[gpu]


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def settings(queries, cache: dict | None = None, gpu: str | None = None):
    """Per-query layers and CTAs per SM from a tuning cache (automatic
    choice for buckets the cache does not cover)."""
    import torch
    q = np.asarray(queries, dtype=np.int64).reshape(-1, 3)
    if cache is None:
        cache = load_cache()
    entry = cache.get(gpu or torch.cuda.get_device_name(), {})
    offs = entry.get("layer_offset", {})
    lgs = []
    for _, n, m in q:
        d = _dims(m)
        lg = auto_log2g(int(n), d) + int(offs.get(bucket(int(n), d), 0))
        lg = max(0, lg)
        while lg > 0 and lg * d > MAX_GRID_BITS:
            lg -= 1
        lgs.append(lg)
    return np.array(lgs, dtype=np.int32), int(entry.get("refine_ctas_per_sm", 0))
