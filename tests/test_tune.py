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


def test_settings_apply_cache_offsets(tmp_path):
    q = np.array([(0, 1000, 0b11), (5, 200000, 0b111111), (9, 50, 0b1)], dtype=np.int64)
    cache = {"FakeGPU": {"layer_offset": {tune.bucket(1000, 2): 1, tune.bucket(200000, 6): -1},
                         "class_ctas": [0, 3, 0, 0], "class_stages": [8, 4, 8, 8], "class_code": [1, 2, 1, 2],
                         "concurrent_classes": 1}}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(cache))
    k = tune.settings(q, tune.load_cache(str(p)), gpu="FakeGPU")
    lgs = k["log2g"]
    assert k["class_ctas"] == [0, 3, 0, 0] and k["class_stages"] == [8, 4, 8, 8]
    assert k["class_code"] == [1, 2, 1, 2] and k["concurrent_classes"] == 1
    assert lgs[0] == tune.auto_log2g(1000, 2) + 1
    assert lgs[1] == tune.auto_log2g(200000, 6) - 1
    assert lgs[2] == tune.auto_log2g(50, 1)
    assert all(int(l) * bin(int(m)).count("1") <= tune.MAX_GRID_BITS for l, (_, _, m) in zip(lgs, q))
    # no entry for this GPU: no knobs (the library defaults apply)
    assert tune.settings(q, cache, gpu="Other") is None
    assert tune.settings(q, {}, gpu="Other") is None


def test_default_knobs_match_the_library_defaults():
    k = tune.default_knobs()
    # fast codes first in the padded-dimension-16 class only, ring depth 8,
    # as many CTAs per SM as fit, classes one after another
    assert k["class_code"] == [1, 1, 1, 2] and k["class_stages"] == [8] * 4
    assert k["class_ctas"] == [0] * 4 and k["concurrent_classes"] == 0
    assert [tune._class(d) for d in (1, 4, 5, 8, 9, 12, 13, 16)] == [0, 0, 1, 1, 2, 2, 3, 3]


def test_layers_leave_invalid_queries_to_the_library():
    # no column, 17 columns: automatic (-1), so that the library rejects them
    q = np.array([(0, 5, 0), (0, 5, 0x1ffff), (0, 100, 0b101)], dtype=np.int64)
    lgs = tune.layers_for(q, {})
    assert lgs[:2].tolist() == [-1, -1] and lgs[2] == tune.auto_log2g(100, 2)
