"""The batched autotuner on the GPU: tune() on a small mixed table and a few
hundred uneven queries, then
* every query's result under the tuned knobs equals the oracle's (tuning
  changes the time, never the result), as do the results under a knob
  setting of every kind (ring depth 4, 7-bit and 3-bit codes in every class,
  few CTAs per SM, concurrent classes);
* the tuned time is not above the library defaults' (the tuner's own
  interleaved measurement, and a fresh one with 10 % allowance for noise);
* Batch applies a cache file's entry for this GPU."""
import json
import statistics

import numpy as np
import pytest

import oracle
import skydata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402
from paper_2107_09993_b300 import tune  # noqa: E402


def _setup():
    # 16 columns, so that queries of every padded-dimension class occur
    T = skydata.mixed_table(400_000, 16, seed=21)
    q = skydata.batched_queries(240, T.shape[0], T.shape[1], seed=22, n_lo=500, n_hi=60_000, d_lo=1, d_hi=16)
    q = np.concatenate([q, np.array([(250_000, 30_000, 0xffff), (210_000, 40_000, 0b111100001111)])])
    tc = torch.from_numpy(T).cuda().t().contiguous().t()
    return T, q, tc


def _check(T, q, res):
    for i, (r0, c, m) in enumerate(q):
        want = oracle.skyline_subset(T, int(r0), int(c), int(m))
        assert res[i].tolist() == want.tolist(), i


def _median_ms(b, reps=5):
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def test_tune_then_results_and_times(tmp_path):
    T, q, tc = _setup()
    cache = tmp_path / "tuning.json"
    entry = tune.tune(tc, q, sample=len(q), per_bucket=4, repeats=2, cache_path=str(cache))
    assert entry["tuned_ms"] <= entry["default_ms"]
    assert entry["candidates"] > 20
    knobs = tune.settings(q, tune.load_cache(str(cache)))
    assert knobs is not None
    b = sky.Batch(tc, q, tuning=knobs)
    b.run()
    _check(T, q, b.results())
    assert np.all(b.query_status() == 0)
    d = sky.Batch(tc, q, tuning=None)
    d.run()
    t_t, t_d = [], []
    for _ in range(3):
        t_t.append(_median_ms(b))
        t_d.append(_median_ms(d))
    assert statistics.median(t_t) <= 1.10 * statistics.median(t_d), (t_t, t_d)
    b.close()
    d.close()


def test_every_knob_kind_keeps_results():
    T, q, tc = _setup()
    for knobs in ({"class_stages": [4, 4, 4, 4], "class_code": [1, 1, 1, 1], "class_ctas": [1, 1, 2, 2]},
                  {"class_stages": [8, 4, 8, 4], "class_code": [2, 2, 2, 2], "concurrent_classes": 1},
                  {"class_ctas": [3, 0, 1, 0], "class_code": [2, 1, 2, 1], "concurrent_classes": 1,
                   "log2g": tune.layers_for(q, {tune.bucket(int(n), bin(int(m)).count("1")): 1
                                                for _, n, m in q})}):
        b = sky.Batch(tc, q, tuning=knobs)
        b.run()
        _check(T, q, b.results())
        b.close()


def test_batch_applies_the_cache_for_this_gpu(tmp_path, monkeypatch):
    T, q, tc = _setup()
    gpu = torch.cuda.get_device_name()
    p = tmp_path / "tuning.json"
    p.write_text(json.dumps({gpu: {"class_code": [2, 2, 2, 2], "class_stages": [4, 4, 4, 4],
                                   "class_ctas": [0, 0, 0, 0], "concurrent_classes": 1, "layer_offset": {}}}))
    monkeypatch.setattr(tune, "DEFAULT_CACHE", str(p))
    monkeypatch.setattr(tune.load_cache, "__defaults__", (str(p),))
    b = sky.Batch(tc, q)
    assert b.tuning is not None and b.tuning["class_code"] == [2, 2, 2, 2] and b.tuning["concurrent_classes"] == 1
    b.run()
    _check(T, q, b.results())
    b.close()
