#!/usr/bin/env python
"""Exact skyline throughput on B300: points/s through the libsky C ABI.

Workload (one "step"): the whole skyline path (steps (a)-(d): map, mark,
prune, refine + compact) over the two large sets of the paper-style
experiments -- n = 10,000,000 anti-correlated points at d = 16 and
n = 10,000,000 independent points at d = 12, float32, seed 1 -- in one
sky_skyline_sets call (the sets run concurrently): 2 * 10^7 input points per
step. Inputs are resident in HBM when the timed region starts; both are
larger than L2 (640 MB and 480 MB), and L2 is also flushed before every timed
step by writing a 512 MB buffer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sky|reference]
    python bench.py --case KIND:N:D[:survivors] [--seed S] [--steps K] [--warmup W]   (one input)
    python bench.py --batched [--steps K] [--warmup W]                  (4,096-query batched workload)

The line also carries: the n = 10^6, d = 8 three-family workload
(`config_1e6x8`), the pruning pass alone on the large sets
(`roofline_prune_large`), the learned proposal against the plain path on its
evaluation sets (`learned_vs_plain`), the 4,096-query batched launch against
plain sky_skyline calls looped over the same queries (`batched_vs_plain`),
and the paper's 3.2e9-point run (`paper_scale`).
N > 1 runs independent replicas (the skyline of one point set is computed on
one GPU), launched under torchrun, weak scaling.
`--impl reference` times the CPU oracle (sort-first skyline) on the host cores
on a bounded row sample of the same workload. The sky arm's line also carries
the paper's own sequential SkyCell (host, one thread) on a smaller sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import skydata  # noqa: E402

SEED = 1
# the step: both large sets (kind, n, d), seed 1
HEADLINE = (("anticorrelated", 10_000_000, 16), ("independent", 10_000_000, 12))
# the n = 10^6, d = 8 workload of the three families (an extra key)
CONFIG_1E6 = (("independent", 1_000_000, 8), ("correlated", 1_000_000, 8), ("anticorrelated", 1_000_000, 8))
METRIC = "skyline input points/s (exact)"
UNIT = "points/s"
# the oracle's bounded sample: the first rows of each headline set
CPU_SAMPLE_ROWS = 50_000
# the paper's largest run: 3.2e9 correlated points, d = 4, layer 6 (Sec. 7).
# Drawn with rows outside the unit cube redrawn instead of clipped: clipping
# piles points onto the faces (x_k = 0), which at 3.2e9 rows gives millions of
# skyline points; the paper's correlated set has 4,203.
PAPER_SCALE = ("correlated_inside", 3_200_000_000, 4)
# pruning pass (steps a-c) measured alone on inputs larger than L2
PRUNE_SETS = (("anticorrelated", 10_000_000, 16), ("independent", 10_000_000, 12))
PRUNE_REPS = 10


def workload_config(extra=None):
    cfg = {"workload": "plain SkyCell, large: n=10,000,000 x d=16 anti-correlated + n=10,000,000 x d=12 "
                       "independent, float32 (seed 1), 2e7 points per step",
           "sets": [{"kind": k, "n": n, "d": d} for k, n, d in HEADLINE], "seed": SEED,
           "l2": "inputs larger than L2 (640 MB, 480 MB); L2 also flushed before every timed step (512 MB write)",
           "options": "default (automatic value map and grid layer)",
           "call": "the step's 2 sets in one sky_skyline_sets call (e2e: sky_skyline_host_sets); the library "
                   "runs them concurrently on internal streams"}
    if extra:
        cfg.update(extra)
    return cfg


def datasets(spec=HEADLINE):
    return [skydata.generate(k, n, d, SEED) for k, n, d in spec]


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        sel = ["-i", gpu_uuid] if gpu_uuid else []
        try:
            self.p = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- roofline --
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def refine_source_hash():
    """Hash of the refinement's source (kernel file and its device body)."""
    return source_hash(("k_refine.cu", "sky_refine.cuh"))


def source_hash(names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2107_09993_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """dram bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get(kernel)
    if not e:
        return None
    if kernel == "k_refine":
        if e.get("source_sha256_16") != refine_source_hash():
            return None
        return e.get("dram_bytes_per_launch")
    if e.get("source_sha256_16") != source_hash(("k_grid.cu", "sky_common.cuh")):
        return None
    return e.get("dram_bytes_per_call")


def ops_per_pair(d):
    # one pair test = ceil(d/4) word subtracts + the AND tree (3-input LOP3) + one compare
    dw = (d + 3) // 4
    return dw + (dw + 1) // 2 + 1


# ------------------------------------------------------------------ sky arm --
def prune_roofline(sky, torch, dev, flush, peaks, peak_src):
    """Steps (a)-(c) alone (survivors_only calls) on the inputs larger than
    L2 that the roofline is quoted on: n = 10^7 anti-correlated at d = 16
    (640 MB) and independent at d = 12 (480 MB), seed 1; L2 evicted before
    every call by their size alone (no flush: both inputs are larger than
    the 126 MB L2, and back-to-back calls leave only the previous call's
    survivor arrays there). Device time of the pruning pass = two CUDA events
    that the library records on its stream around the call's kernel sequence
    (clear, value-map parameters, map + mark, prefix-OR, survivor flags +
    scatter, which writes the ids straight into the caller's buffer),
    replayed as a CUDA graph. `call_ms` is the whole call as the caller sees it (CUDA events on
    the calling stream around sky_skyline, graph replay, host launch and the
    count read-back included). Algorithmic bytes per call: 4nd (map read)
    + 16n (cell and Morton keys written and read) + 8m (survivor keys and
    ids written)."""
    stream = torch.cuda.current_stream(dev)
    per_set = {}
    tot_b, tot_ms = 0, 0.0
    tot_bs, tot_ms_g = 0, 0.0
    phases = ("normalize_ms", "map_mark_ms", "prune_ms", "survivors_ms")
    for kind, n, d in PRUNE_SETS:
        x = torch.from_numpy(skydata.generate(kind, n, d, SEED)).to(dev)
        out = torch.empty(n, dtype=torch.int32, device=dev)
        for _ in range(3):
            sky.skyline(x, survivors_only=True, out=out)
        calls = []
        for _ in range(PRUNE_REPS):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sky.skyline(x, survivors_only=True, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            calls.append(e0.elapsed_time(e1))
        # device time of the call's kernel sequence (graph replay), then the
        # per-phase split (kernels launched one by one: adds launch gaps)
        sky.set_phase_timing(2)
        sky.skyline(x, survivors_only=True, out=out)
        dev_ms = []
        for _ in range(PRUNE_REPS):
            torch.cuda.synchronize(dev)
            sky.skyline(x, survivors_only=True, out=out)
            dev_ms.append(sky.last_phase_times()["call_ms"])
        sky.set_phase_timing(1)
        sky.skyline(x, survivors_only=True, out=out)
        by_phase = {k: [] for k in phases}
        for _ in range(PRUNE_REPS):
            torch.cuda.synchronize(dev)
            sky.skyline(x, survivors_only=True, out=out)
            ph = sky.last_phase_times()
            for k in phases:
                by_phase[k].append(ph[k])
        st = sky.last_run_stats()
        # the survivor layout of step (d): k_gather writes the compacted
        # survivor coordinates (Morton order) after the sort; timed with
        # phase events in full calls
        full = torch.empty(n, dtype=torch.int32, device=dev)
        sky.skyline(x, out=full)
        gat = []
        for _ in range(3):
            torch.cuda.synchronize(dev)
            sky.skyline(x, out=full)
            gat.append(sky.last_phase_times()["gather_ms"])
        del full
        sky.set_phase_timing(False)
        m = st["survivors"]
        b = 4 * n * d + 16 * n + 8 * m
        # the pruning pass's bytes as the method needs them: read the points,
        # re-read them or a 4-byte key per point, write the compacted
        # survivors (coordinates + id)
        b_survey = 4 * n * d + min(4 * n * d, 8 * n) + m * (4 * d + 4)
        med = statistics.median(dev_ms)
        g_ms = statistics.median(gat)
        per_set[f"{kind} n={n} d={d}"] = {
            "ms": round(med, 4), "call_ms": round(statistics.median(calls), 4), "survivors": m,
            "log2_g": st["log2_g"], "gbs": round(b / (med / 1e3) / 1e9, 1),
            "phase_ms_direct_launches": {k: round(statistics.median(v), 4) for k, v in by_phase.items()},
            "gather_ms": round(g_ms, 4),
            "method_bytes": b_survey,
            "method_gbs_pass_plus_gather": round(b_survey / ((med + g_ms) / 1e3) / 1e9, 1)}
        tot_b += b
        tot_ms += med
        tot_bs += b_survey
        tot_ms_g += med + g_ms
        del x, out
    gbs = tot_b / (tot_ms / 1e3) / 1e9
    # DRAM bytes per call of the same kernels from the committed ncu capture
    # (mean of the two sets), if the pruning kernels are unchanged since
    tr = profiled_traffic("pruning_pass")
    traffic = None
    if tr and all(f"{k} n={n} d={d}" in tr for k, n, d in PRUNE_SETS):
        traffic = int(sum(tr[f"{k} n={n} d={d}"] for k, n, d in PRUNE_SETS) / len(PRUNE_SETS))
        for k, n, d in PRUNE_SETS:
            per_set[f"{k} n={n} d={d}"]["traffic"] = tr[f"{k} n={n} d={d}"]
    return {"kernel": "pruning pass: k_clear, k_sample_params, k_map_mark_tma (+ k_occ_merge), "
                      "k_prefix_low/high, k_surv_flags, k_surv_scatter",
            "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(gbs / peaks["hbm_gbs"], 4),
            "frac_of_nominal_8000": round(gbs / 8000.0, 4),
            "traffic": traffic,
            "algorithmic_bytes_per_call": int(tot_b / len(PRUNE_SETS)),
            "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json)" if peak_src == "measured"
            else "fallback 6.4 TB/s",
            "timing": "device time of the pass: two CUDA events on the library's stream around the call's "
                      "kernel sequence (CUDA-graph replay, sky_set_phase_timing(2)), median of the calls",
            "method_bytes_view": {
                "bytes": "4nd + min(4nd, 8n) + m(4d + 4): read the points, re-read a 4-byte key per point, write "
                         "the m compacted survivors (coordinates + id)",
                "time": "the pass plus k_gather, which writes the survivor coordinates after the Morton sort",
                "achieved": round(tot_bs / (tot_ms_g / 1e3) / 1e9, 1),
                "frac": round(tot_bs / (tot_ms_g / 1e3) / 1e9 / peaks["hbm_gbs"], 4),
                "frac_of_nominal_8000": round(tot_bs / (tot_ms_g / 1e3) / 1e9 / 8000.0, 4)},
            "workload": "; ".join(f"{k} n={n:,} d={d}" for k, n, d in PRUNE_SETS)
                        + f" (seed {SEED}); median of {PRUNE_REPS} calls each; inputs larger than L2, no flush",
            "per_set": per_set}


def paper_scale(sky, torch, dev):
    """The paper's largest workload on one B300: 3.2e9 correlated points,
    d = 4, drawn on the device (skydata.generate_torch, seed 1), skyline by
    sky_skyline_chunked from device memory (the automatic layer is 6, the
    paper's rho). Median of 3 calls after one warm-up, CUDA events."""
    kind, n, d = PAPER_SCALE
    need = n * d * 4 + (16 << 30)
    free, _ = torch.cuda.mem_get_info(dev)
    if free < need:
        return {"skipped": f"needs about {need / 2**30:.0f} GiB free device memory, {free / 2**30:.0f} GiB free"}
    x = skydata.generate_torch(kind, n, d, SEED, device=dev)
    r = sky.skyline_chunked(x)
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = sky.skyline_chunked(x)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    st = sky.last_run_stats()
    med = statistics.median(ms)
    del x
    torch.cuda.empty_cache()
    return {"workload": f"{kind} n={n:,} d={d}, device-resident, drawn on the GPU (seed {SEED})",
            "ms": round(med, 2), "points_per_s": round(n / (med / 1e3), 1), "skyline": int(r.numel()),
            "candidates_after_step_c": st["n"], "log2_g_refine": st["log2_g"],
            "paper": {"seconds": 0.6, "points_per_s": 5.3e9, "skyline": 4203,
                      "hardware": "Quadro RTX 6000 (Turing, 24 GB); its generator and timing boundaries differ"}}


def time_step(fn, stream, dev, flush=None):
    """Device time of one call of fn (CUDA events on `stream`), ms."""
    import torch
    if flush is not None:
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1), out


def config_1e6(sky, torch, dev, flush, steps):
    """The n = 10^6, d = 8 workload (independent, correlated, anti-correlated,
    seed 1) as one sky_skyline_sets call per step, L2 flushed before each."""
    xs = [torch.from_numpy(P).to(dev) for P in datasets(CONFIG_1E6)]
    outs = [torch.empty(x.shape[0], dtype=torch.int32, device=dev) for x in xs]
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        sky.skyline_sets(xs, outs=outs)
    ms = [time_step(lambda: sky.skyline_sets(xs, outs=outs), stream, dev, flush)[0] for _ in range(steps)]
    _, res = time_step(lambda: sky.skyline_sets(xs, outs=outs), stream, dev, flush)
    med = statistics.median(ms)
    pts = sum(n for _, n, _ in CONFIG_1E6)
    return {"workload": "n=1,000,000 x d=8 float32, independent + correlated + anti-correlated (seed 1), "
                        "one sky_skyline_sets call, L2 flushed", "ms_per_step": round(med, 4),
            "points_per_s": round(pts / (med / 1e3), 1), "skyline_sizes": [int(r.numel()) for r in res],
            "steps": steps}


def learned_vs_plain(sky, torch, dev, reps=5):
    """The learned proposal's evaluation sets (Gaussian copula, n = 10^7,
    d = 8, seed 3, rho in {-0.8, 0, 0.8}): the plain path (automatic layer)
    against the learned path (sky_propose with the shipped weights, then
    sky_skyline with the proposed layer and the 16 filter points), both
    device-resident, median of `reps` calls each after a warm-up; the index
    sets must be identical."""
    from paper_2107_09993_b300 import learned
    params, meta = learned.load_weights(device=str(dev))
    n_ref = int(meta["rows_per_set"])
    stream = torch.cuda.current_stream(dev)
    out = {}
    for rho in (-0.8, 0.0, 0.8):
        P, rho_eff = skydata.copula(10_000_000, 8, 3, rho)
        x = torch.from_numpy(P).to(dev)
        del P
        plain = lambda: sky.skyline(x)                                    # noqa: E731
        learn = lambda: sky.skyline_learned(x, params, n_ref=n_ref)       # noqa: E731
        for _ in range(2):
            plain()
            learn()
        tp, a = [], None
        for _ in range(reps):
            t, a = time_step(plain, stream, dev)
            tp.append(t)
        sp = sky.last_run_stats()
        tl, b = [], None
        for _ in range(reps):
            t, b = time_step(learn, stream, dev)
            tl.append(t)
        sl = sky.last_run_stats()
        mp, ml = statistics.median(tp), statistics.median(tl)
        out[f"rho={rho:+.1f}"] = {"rho_eff": round(rho_eff, 4), "plain_ms": round(mp, 3), "learned_ms": round(ml, 3),
                                  "speedup": round(mp / ml, 3), "identical": bool(torch.equal(a, b)),
                                  "skyline": int(a.numel()), "survivors_plain": sp["survivors"],
                                  "survivors_learned": sl["survivors"], "log2_g_plain": sp["log2_g"],
                                  "log2_g_learned": sl["log2_g"], "n_filter_used": sl["n_filter_used"]}
        del x
    return {"workload": "Gaussian copula n=10,000,000 x d=8 float32 (seed 3), rho in {-0.8, 0, 0.8}",
            "timing": f"device time per call (CUDA events, host launch included), median of {reps}; the learned "
                      "time includes sky_propose (features + network + decode)",
            "sets": out}


def batched_vs_plain(sky, torch, dev, reps=3):
    """The batched workload: 4,096 queries (row count log-uniform in
    [1e3, 1e6], d uniform in {2..12}, random column subsets and row ranges;
    seed 2) on a 20M x 12 float32 table, half independent and half
    anti-correlated, stored column-major on the device. Batched: one
    sky_skyline_batched launch (CUDA graph). Plain: sky_skyline looped over
    the same 4,096 queries on one stream, each query's rows and columns
    gathered into its own contiguous input and its output buffer allocated
    before the timed loop, so only the sky_skyline calls are timed. Results
    compared query by query."""
    import numpy as np
    n_rows, n_cols, nq = 20_000_000, 12, 4096
    T = skydata.mixed_table(n_rows, n_cols, seed=2)
    q = skydata.batched_queries(nq, n_rows, n_cols, seed=2)
    t = torch.from_numpy(T).to(dev)
    del T
    tc = t.t().contiguous().t()
    stream = torch.cuda.current_stream(dev)
    # library defaults, then the autotuner's cached choices for this GPU
    # (tune.py; Batch applies them by default)
    b0 = sky.Batch(tc, q, tuning=None)
    for _ in range(2):
        b0.run()
    mb0 = [time_step(b0.run, stream, dev)[0] for _ in range(reps)]
    b0.close()
    b = sky.Batch(tc, q)
    tuned = b.tuning is not None
    for _ in range(2):
        b.run()
    mb = [time_step(b.run, stream, dev)[0] for _ in range(reps)]
    st = b.stats()
    bres = b.results()
    bad = int((b.query_status() != 0).sum())
    knobs = {k: v for k, v in (b.tuning or {}).items() if k != "log2g"}
    b.close()
    # the same queries planned on the device (sky_skyline_batched_device):
    # records in device memory, bound-sized grids, library default variants
    qd = torch.as_tensor(np.asarray(q, dtype=np.int64)).to(dev)
    rec = sky.query_records(qd[:, 0], qd[:, 1], qd[:, 2])
    db = sky.DeviceBatch(tc, nq, int(q[:, 1].sum()))
    for _ in range(2):
        db.run(rec)
    md = [time_step(lambda: db.run(rec), stream, dev)[0] for _ in range(reps)]
    dres = db.results()
    dsame = all(np.array_equal(x, y) for x, y in zip(dres, bres)) and bool((db.query_status() == 0).all())
    del db, dres, rec, qd
    del tc
    subs, outs = [], []
    for (r0, c, m) in q:
        cols = [k for k in range(n_cols) if (int(m) >> k) & 1]
        subs.append(t[int(r0):int(r0) + int(c)][:, cols].contiguous())
        outs.append(torch.empty(int(c), dtype=torch.int32, device=dev))
    del t

    def loop():
        return [sky.skyline(x, out=o) for x, o in zip(subs, outs)]

    loop()
    ml = []
    res = None
    for _ in range(reps):
        ms, res = time_step(loop, stream, dev)
        ml.append(ms)
    same = all(np.array_equal(r.cpu().numpy() + int(q[i, 0]), bres[i]) for i, r in enumerate(res))
    del subs, outs, res
    torch.cuda.empty_cache()
    pts = int(q[:, 1].sum())
    mbm, mlm = statistics.median(mb), statistics.median(ml)
    return {"workload": "batched: 4,096 queries on a 20M x 12 mixed table (seed 2), column-major",
            "tuning": {"applied": tuned, "source": "paper_2107_09993_b300/tuning.json (tune.py, this GPU's entry)",
                       "knobs": knobs, "batched_default_ms": round(statistics.median(mb0), 2)},
            "device_planned": {"ms": round(statistics.median(md), 2), "identical": dsame,
                               "what": "sky_skyline_batched_device: queries in device memory, planned by a kernel, "
                                       "no host round trip (default variants)"},
            "points": pts, "batched_ms": round(mbm, 2), "looped_plain_ms": round(mlm, 2),
            "speedup": round(mlm / mbm, 3), "batched_points_per_s": round(pts / (mbm / 1e3), 1),
            "identical": bool(same), "query_errors": bad, "skyline": st["skyline"], "survivors": st["survivors"],
            "timing": f"median of {reps}: one graph launch vs 4,096 sky_skyline calls (inputs gathered and outputs "
                      "allocated before the timed loop); CUDA events on the calling stream"}


def tournament_vs_prefix_or(sky, torch, dev, reps=3):
    """Step (c)'s classes by the paper's tournament tree (Algorithm 3, one
    kernel per tree level, d passes; sky_tournament_cells) on the occupancy
    of the large sets' layers, against the prefix-OR path's step (c) on the
    same grid (sky_prune_cells: prefix-OR + dominated bitmap + survivors,
    Grid API). Device time, median of `reps`; the dominated cells of the two
    must be equal."""
    import numpy as np
    stream = torch.cuda.current_stream(dev)
    out = {}
    for kind, n, d in (("anticorrelated", 10_000_000, 16), ("independent", 10_000_000, 12),
                       ("anticorrelated", 1_000_000, 8)):
        x = torch.from_numpy(skydata.generate(kind, n, d, SEED)).to(dev)
        g = sky.Grid(x)
        g.prune()
        lg = g.stats()["log2_g"]
        occ = g.occupied()
        dom = g.dominated()
        t_pre = []
        for _ in range(reps):
            g2 = sky.Grid(x, log2_g=lg)
            torch.cuda.synchronize(dev)
            ms, _ = time_step(lambda: g2.prune(), stream, dev)
            t_pre.append(ms)
            g2.close()
        t_tt = []
        cls = None
        for _ in range(reps):
            ms, cls = time_step(lambda: sky.tournament_cells(occ, d, lg), stream, dev)
            t_tt.append(ms)
        ncell = 1 << (lg * d)
        w = dom.cpu().numpy().view(np.uint32)
        want = ((w[np.arange(ncell) >> 5] >> (np.arange(ncell) & 31).astype(np.uint32)) & 1).astype(np.uint8)
        got = (cls.cpu().numpy() & 1).astype(np.uint8)
        out[f"{kind} n={n} d={d}"] = {"log2_g": lg, "cells": ncell,
                                      "tournament_ms": round(statistics.median(t_tt), 3),
                                      "prefix_or_prune_ms": round(statistics.median(t_pre), 3),
                                      "tournament_launches": d * (2 * lg * d + 3) + 1,
                                      "dominated_equal": bool(np.array_equal(got, want)),
                                      "key_cells": int(((cls >> 1) & 1).sum().item()),
                                      "candidate_cells": int(((cls >> 2) & 1).sum().item())}
        g.close()
        del x
    return {"what": "step (c) classes: the paper's tournament tree (Algorithm 3, as read: all cells are leaves, "
                    "one dimension per pass) vs this library's prefix-OR path on the same layer",
            "timing": f"CUDA events on the calling stream around each call (host launches included), median of {reps}",
            "sets": out}


def run_sky(args):
    import torch
    import paper_2107_09993_b300 as sky

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    host = datasets()
    xs = [torch.from_numpy(P).to(dev) for P in host]
    outs = [torch.empty(P.shape[0], dtype=torch.int32, device=dev) for P in host]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step():
        # the step's sets in one call: they run concurrently
        return [int(r.numel()) for r in sky.skyline_sets(xs, outs=outs)]

    for _ in range(args.warmup):
        step()
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    clocks = ClockSampler(uuid) if rank == 0 else None
    time.sleep(0.5)   # let the sampler start before the timed region
    # ---- timed region: K steps, L2 flushed before each, device-resident inputs
    total_ms = 0.0
    launches = 0
    sizes = None
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sizes = step()
        launches += sky.last_run_stats()["kernels"]   # summed over the sets
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
    barrier()
    clk = clocks.stop() if clocks else None
    # ---- per-phase times: the step's sets again, one sky_skyline call at a
    # time, with CUDA events recorded between the phases on the library's
    # stream (direct launches)
    sky.set_phase_timing(True)
    phase_sum = {}
    ops = 0
    pairs = 0
    b_prune = 0
    phase_steps = max(1, min(args.steps, 5))
    for _ in range(phase_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        for x, o in zip(xs, outs):
            sky.skyline(x, out=o)
            st = sky.last_run_stats()
            ph = sky.last_phase_times()
            pairs += st["pairs"]
            ops += st["pairs"] * ops_per_pair(st["d"])
            n, d, m = st["n"], st["d"], st["survivors"]
            # map read + (cell, Morton) key write/read + (Morton, id) write
            b_prune += 4 * n * d + 16 * n + 8 * m
            for k, v in ph.items():
                phase_sum[k] = phase_sum.get(k, 0.0) + v
    sky.set_phase_timing(False)

    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max_ms = float(t.item())
    pts_per_step = sum(P.shape[0] for P in host)
    value = world * args.steps * pts_per_step / (t_max_ms / 1e3)

    # ---- end to end through the host-buffer entry point (pinned memory)
    pinned = [torch.from_numpy(P).pin_memory() for P in host]
    hout = [torch.empty(P.shape[0], dtype=torch.int32).pin_memory() for P in host]
    for _ in range(max(args.warmup, 2)):   # the second call captures the graphs
        sky.skyline_host_sets(pinned, outs=hout)
    e2e_ms = 0.0
    d2h = 0
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        d2h = 0
        for r in sky.skyline_host_sets(pinned, outs=hout):
            d2h += 4 * int(r.numel()) + 8
        e2e_ms += (time.perf_counter() - t0) * 1e3
    barrier()
    del pinned, hout
    te = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * args.steps * pts_per_step / (float(te.item()) / 1e3)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1900.0
    # dominant kernel: the phase with the largest device time
    dom_phase = max(phase_sum, key=phase_sum.get)
    refine_s = phase_sum["refine_ms"] / 1e3
    alu_peak_gops = 148 * 128 * sm_mhz * 1e6 / 1e9  # int32 lane ops/s, measured median SM clock
    refine_gops = ops / refine_s / 1e9 if refine_s > 0 else 0.0
    prune_s = (phase_sum["normalize_ms"] + phase_sum["map_mark_ms"] + phase_sum["prune_ms"]
               + phase_sum["survivors_ms"]) / 1e3
    prune_gbs = b_prune / prune_s / 1e9 if prune_s > 0 else 0.0
    launches_refine = phase_steps * len(HEADLINE)
    traffic = profiled_traffic("k_refine")
    roof_refine = {"kernel": "k_refine", "bound": "alu", "achieved": round(refine_gops, 1),
                   "peak": round(alu_peak_gops, 1), "unit": "Gop/s",
                   "frac": round(refine_gops / alu_peak_gops, 4),
                   "traffic": traffic,
                   "peak_source": f"148 SMs x 128 int32 lanes x {sm_mhz:.0f} MHz (median SM clock sampled during the run)",
                   "work": f"{pairs / launches_refine:.4g} candidate pair tests per launch x ops per test "
                           f"(ceil(d/4) word subtracts + AND tree + compare: 7 at d = 16, 6 at d = 12; the work "
                           f"measure of the list probe, kept for the mask probe that tests these pairs from "
                           f"padded dimension 12, 32 per lane with d table loads and ANDs)",
                   "ms_per_launch": round(phase_sum['refine_ms'] / launches_refine, 4),
                   "timing": "per set: the refinement phase (phase events, direct launches) -- from 2^21 rows "
                             "two k_refine launches (pre-pass, full pass) with the compaction, the second gather "
                             "and the p-tile ordering between them; pair tests of both launches counted"}
    roof_prune = {"kernel": "pruning pass (phases map + prune + survivors of the timed workload)",
                  "bound": "hbm", "achieved": round(prune_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": round(prune_gbs / peaks["hbm_gbs"], 4), "traffic": None,
                  "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json)" if peak_src == "measured"
                  else "fallback 6.4 TB/s",
                  "note": "phase events between direct launches (host gaps included); roofline_prune_large "
                          "times the same pass as one graph replay"}
    roofline = roof_refine if dom_phase == "refine_ms" else roof_prune
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (skydata generators, seed 1)",
        "config": workload_config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                "h2d_bytes_per_step": sum(int(P.nbytes) for P in host), "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_prune": roof_prune,
        "phase_ms_per_step": {k: round(v / phase_steps, 4) for k, v in phase_sum.items()},
        "skyline_sizes": sizes,
        "clocks": clk,
    }
    del xs, outs
    torch.cuda.empty_cache()
    if not args.no_extras:
        line["config_1e6x8"] = config_1e6(sky, torch, dev, flush, max(args.steps, 10))
        line["roofline_prune_large"] = prune_roofline(sky, torch, dev, flush, peaks, peak_src)
        line["learned_vs_plain"] = learned_vs_plain(sky, torch, dev)
        line["batched_vs_plain"] = batched_vs_plain(sky, torch, dev)
        line["tournament_vs_prefix_or"] = tournament_vs_prefix_or(sky, torch, dev)
        line["paper_scale"] = paper_scale(sky, torch, dev)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(host, args.cpu_seconds)
        line["cpu_baseline_sequential"] = seq_baseline(datasets(CONFIG_1E6), args.cpu_seconds / 2)
        line["cpu_oracle_full_sets"] = oracle_full_times()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------- CPU baseline --
def cpu_sample_step(host, rows):
    import oracle
    t0 = time.perf_counter()
    for P in host:
        oracle.skyline_sfs(P[:rows])
    return time.perf_counter() - t0


def cpu_baseline(host, seconds):
    import oracle
    rows = CPU_SAMPLE_ROWS
    spent, reps = 0.0, 0
    while spent < seconds or reps == 0:
        spent += cpu_sample_step(host, rows)
        reps += 1
    value = reps * rows * len(host) / spent
    return {"value": round(value, 1), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"sort-first skyline oracle on the first {rows:,} rows of each of the {len(host)} sets of "
                      f"the step, {reps} repetition(s), {spent:.1f} s (its cost grows with n x |skyline|, so "
                      "the full sets run far slower per point: see cpu_oracle_full_sets)"}


def oracle_full_times():
    """The oracle on whole sets, as recorded when tests/golden/make_fullsize.py
    wrote the parity hashes (build host, not this box): context only."""
    p = os.path.join(ROOT, "tests", "golden", "fullsize_oracle.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        g = json.load(f)["sets"]
    out = {k: {"n": v["n"], "d": v["d"], "skyline": v["count"], "seconds": v["oracle_seconds"],
               "threads": v["threads"], "points_per_s": round(v["n"] / v["oracle_seconds"], 1)}
           for k, v in g.items() if v.get("oracle_seconds")}
    out["note"] = ("build host, not the GPU box; the anti-correlated 10^7 x 16 set (8.2e6 skyline points) was not "
                   "run: the oracle's cost grows with the square of the skyline (days)")
    return out


SEQ_SAMPLE_ROWS = 20_000


def seq_baseline(host, seconds):
    """The paper's sequential SkyCell on the host (one thread), on the first
    SEQ_SAMPLE_ROWS rows of each n = 10^6 x 8 dataset, repeated for about
    `seconds`."""
    import paper_2107_09993_b300 as sky
    rows = SEQ_SAMPLE_ROWS
    spent, reps = 0.0, 0
    while spent < seconds or reps == 0:
        t0 = time.perf_counter()
        for P in host:
            sky.baseline_sequential(P[:rows])
        spent += time.perf_counter() - t0
        reps += 1
    value = reps * rows * len(host) / spent
    return {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "paper's sequential SkyCell (Alg. 1 + 2)",
            "sample": f"first {rows:,} rows of each of the 3 n=10^6 x d=8 sets, {reps} repetition(s), {spent:.1f} s"}


# -------------------------------------------------------------- reference --
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    host = datasets()
    rows = CPU_SAMPLE_ROWS
    for _ in range(args.warmup):
        cpu_sample_step(host, rows // 10)
    t = 0.0
    for _ in range(args.steps):
        t += cpu_sample_step(host, rows)
    value = args.steps * rows * len(host) / t
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (skydata generators, seed 1)",
        "config": workload_config({"sample": f"first {rows:,} rows of each set per step"}),
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"first {rows:,} rows of each of the {len(host)} sets per step"},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_case(args):
    """One named input (for profiling runs): `--case KIND:N:D[:survivors]`
    runs `warmup` untimed and `steps` timed sky_skyline calls on the seeded
    set and prints one JSON line with their median time and the run stats."""
    import torch
    import paper_2107_09993_b300 as sky

    parts = args.case.split(":")
    kind, n, d = parts[0], int(parts[1]), int(parts[2])
    surv = len(parts) > 3 and parts[3] == "survivors"
    x = torch.from_numpy(skydata.generate(kind, n, d, args.seed)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        sky.skyline(x, survivors_only=surv, out=out)
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sky.skyline(x, survivors_only=surv, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"case": args.case, "seed": args.seed, "calls": args.steps,
                      "ms_median": round(statistics.median(ms), 4) if ms else None,
                      "stats": sky.last_run_stats()}), flush=True)


def run_batched(args):
    """The batched workload: 4,096 skyline queries (row count log-uniform in
    [1e3, 1e6], d uniform in {2..12}, random column subsets and row ranges) on
    a 20M x 12 float32 table, half independent and half anti-correlated
    (seed 2), stored column-major on the device. One CUDA-graph launch per
    step; `steps` timed launches after `warmup`. Reference point: the same
    first 256 queries as plain sky_skyline calls in a loop (columns gathered
    per query) against one batched launch of those 256. One JSON line."""
    import torch
    import paper_2107_09993_b300 as sky

    n_rows, n_cols, nq = 20_000_000, 12, 4096
    T = skydata.mixed_table(n_rows, n_cols, seed=2)
    q = skydata.batched_queries(nq, n_rows, n_cols, seed=2)
    t = torch.from_numpy(T).cuda()
    tc = t.t().contiguous().t()
    b = sky.Batch(tc, q)
    for _ in range(args.warmup):
        b.run()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = b.stats()
    bad = int((b.query_status() != 0).sum())
    b.close()
    sel = q[:256]
    b2 = sky.Batch(tc, sel)
    b2.run()
    ms_b = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b2.run()
        e1.record()
        torch.cuda.synchronize()
        ms_b.append(e0.elapsed_time(e1))
    b2.close()
    ms_l = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (r0, c, m) in sel:
            cols = [k for k in range(n_cols) if (int(m) >> k) & 1]
            sky.skyline(t[int(r0):int(r0) + int(c)][:, cols].contiguous())
        torch.cuda.synchronize()
        ms_l.append((time.perf_counter() - t0) * 1e3)
    med = statistics.median(ms)
    pts = int(q[:, 1].sum())
    print(json.dumps({
        "workload": "batched: 4,096 queries on a 20M x 12 mixed table (seed 2), one graph launch",
        "points": pts, "ms_per_launch": round(med, 2), "points_per_s": round(pts / (med / 1e3), 1),
        "skyline": st["skyline"], "survivors": st["survivors"], "query_errors": bad,
        "first_256": {"batched_ms": round(min(ms_b), 2), "looped_plain_ms": round(min(ms_l), 2),
                      "speedup": round(min(ms_l) / min(ms_b), 2)}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sky", "reference"], default="sky")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the large-input pruning roofline and the paper-scale run (launch-list profiling)")
    ap.add_argument("--batched", action="store_true", help="time the batched workload (4,096 queries) only")
    ap.add_argument("--seed", type=int, default=SEED, help="seed of the --case input")
    ap.add_argument("--case", default=None,
                    help="KIND:N:D[:survivors] -- time one seeded input only (profiling runs)")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_sky(args)


if __name__ == "__main__":
    main()
