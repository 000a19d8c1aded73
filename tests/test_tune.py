"""CPU checks of the batched autotuner's host logic (buckets, cache use)."""
import json

import numpy as np

from paper_2107_09993_b300 import tune


def test_auto_layer_rule_and_limits():
    for n in (10, 1000, 10 ** 6):
        for d in range(1, 17):
            lg = tune.auto_log2g(n, d)
            assert lg >= 1 and lg * d <= max(tune.MAX_GRID_BITS, d)
    assert tune.auto_log2g(10 ** 6, 8) == 2         # 24 bits would exceed the batched 2^18 cells
    assert tune.auto_log2g(10 ** 6, 2) == 8         # the automatic layer stops at 8 (256 columns)
    assert tune.auto_log2g(10 ** 6, 3) == 6         # 18 bits: the batched limit


def test_settings_apply_cache_offsets(tmp_path, monkeypatch):
    q = np.array([(0, 1000, 0b11), (5, 200000, 0b111111), (9, 50, 0b1)], dtype=np.int64)
    cache = {"FakeGPU": {"layer_offset": {tune.bucket(1000, 2): 1, tune.bucket(200000, 6): -1},
                         "refine_ctas_per_sm": 3}}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(cache))
    lgs, ctas = tune.settings(q, tune.load_cache(str(p)), gpu="FakeGPU")
    assert ctas == 3
    assert lgs[0] == tune.auto_log2g(1000, 2) + 1
    assert lgs[1] == tune.auto_log2g(200000, 6) - 1
    assert lgs[2] == tune.auto_log2g(50, 1)
    assert all(int(l) * bin(int(m)).count("1") <= tune.MAX_GRID_BITS for l, (_, _, m) in zip(lgs, q))
    lgs2, ctas2 = tune.settings(q, {}, gpu="Other")
    assert ctas2 == 0 and lgs2[0] == tune.auto_log2g(1000, 2)
