"""The shipped proposal weights (CPU): shape, bit patterns and training
record, and the layer shift that carries a prediction to another set size."""
import json
import os

import numpy as np

from oracle import mlp as omlp
from paper_2107_09993_b300 import learned


def test_shipped_weights_file():
    z = np.load(learned.WEIGHTS, allow_pickle=False)
    bits = z["bf16"]
    assert bits.dtype == np.uint16 and bits.shape == (omlp.n_params(),)
    w = (bits.astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isfinite(w)) and np.abs(w).max() < 64
    meta = json.loads(str(z["meta"]))
    assert meta["sets"] == 10000 and meta["rows_per_set"] == 100000
    assert meta["held_out_layer_accuracy"] > 0.7
    assert os.path.getsize(learned.WEIGHTS) < 200_000


def test_automatic_layer_rule():
    # largest log2_g <= min(8, 24 / d) with 2^(log2_g * d) <= 32 n
    assert [learned.auto_layer(100_000, d) for d in (2, 3, 4, 8, 16)] == [8, 7, 5, 2, 1]
    assert [learned.auto_layer(10_000_000, d) for d in (2, 3, 4, 8, 16)] == [8, 8, 6, 3, 1]
    for n in (1, 1000, 10**6, 10**9):
        for d in range(1, 17):
            r = learned.auto_layer(n, d)
            assert 1 <= r <= max(1, min(8, 24 // d))
            assert r == 1 or (1 << (r * d)) <= 32 * n
            assert r == min(8, 24 // d) or (1 << ((r + 1) * d)) > 32 * n
