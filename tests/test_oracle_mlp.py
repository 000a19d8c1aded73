"""Pins for the learned proposal's oracle (oracle/mlp.py).

Fixed by the mathematics: finite differences for every parameter group,
closed-form losses, the first AdamW step, exact bfloat16 roundings, and
features of constructed datasets with known histograms and correlations.
"""
import numpy as np

from oracle import mlp


def _rand_problem(rng, B=3):
    theta = rng.normal(0, 0.3, mlp.n_params())
    F = rng.random((B, mlp.F_IN))
    d = rng.integers(2, 17, size=B)
    labels = np.array([int(rng.integers(0, min(8, 24 // di))) for di in d])
    targets = rng.random((B, mlp.N_FILT * mlp.DMAX))
    masks = np.zeros_like(targets)
    for i, di in enumerate(d):
        masks[i].reshape(mlp.N_FILT, mlp.DMAX)[:, :di] = 1
    return theta, F, d, labels, targets, masks


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta, F, d, labels, targets, masks = _rand_problem(rng)
    L, G = mlp.batch_loss_grad(theta, F, d, labels, targets, masks, lam=0.7)
    # probe coordinates of every parameter group
    starts = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    probes = []
    for a, b in zip(starts[:-1], starts[1:]):
        probes += list(rng.choice(np.arange(a, b), size=6, replace=False))
    h = 1e-6
    for i in probes:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        num = (mlp.batch_loss_grad(tp, F, d, labels, targets, masks, 0.7)[0]
               - mlp.batch_loss_grad(tm, F, d, labels, targets, masks, 0.7)[0]) / (2 * h)
        assert abs(num - G[i]) <= 1e-6 + 1e-4 * abs(num), (i, num, G[i])


def test_loss_closed_forms():
    y = np.zeros(mlp.OUT)
    t = np.zeros(mlp.N_FILT * mlp.DMAX)
    m = np.ones_like(t)
    for d in (2, 3, 8, 16):
        L, dy = mlp.loss(y, d, 0, t, m, lam=1.0)
        nv = mlp.valid_layers(d).sum()
        assert nv == 24 // d if d >= 3 else nv == 8
        assert np.isclose(L, np.log(nv))                    # uniform logits, zero residual
        assert np.isclose(dy[:mlp.N_LAYERS].sum(), 0.0)
        assert np.all(dy[mlp.N_LAYERS:][m > 0] == 0)
    y2 = y.copy()
    y2[mlp.N_LAYERS:] = 0.5
    L2, _ = mlp.loss(y2, 16, 0, t, m, lam=2.0)
    assert np.isclose(L2 - np.log(1), 2.0 * 0.25)           # d = 16: one admissible layer


def test_first_adamw_step():
    rng = np.random.default_rng(1)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    th2, m, v = mlp.adamw(th, g, np.zeros(50), np.zeros(50), step=1, lr=1e-2, wd=0.1)
    assert np.allclose(th2, th - 1e-2 * (g / (np.abs(g) + 1e-8) + 0.1 * th))


def test_bf16_rounding():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3.0e38], dtype=np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even
    assert r[2] == np.float32(1 + 2 ** -6)  # tie -> even (up)
    assert r[3] == np.float32(1 + 2 ** -7)  # representable
    assert r[4] == -2.5
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


def test_features_of_constructed_data():
    n = 32 * 100
    base = (np.arange(n) % 32 + 0.5) / 32.0      # every bin equally filled
    P = np.stack([base, base, 1.0 - base, np.sin(np.arange(n))], axis=1).astype(np.float32)
    f = mlp.features(P)
    hist = f[:mlp.DMAX * mlp.BINS].reshape(mlp.DMAX, mlp.BINS)
    assert np.allclose(hist[0], 1 / 32) and np.allclose(hist[2], 1 / 32)
    assert np.allclose(hist[4:], 0)
    tri = f[mlp.DMAX * mlp.BINS: mlp.DMAX * mlp.BINS + 120]
    idx = {(k, l): i for i, (k, l) in enumerate((k, l) for k in range(16) for l in range(k + 1, 16))}
    assert np.isclose(tri[idx[(0, 1)]], 1.0)
    assert np.isclose(tri[idx[(0, 2)]], -1.0)
    assert abs(tri[idx[(0, 3)]]) < 0.1
    assert np.allclose([tri[idx[(k, l)]] for k in range(16) for l in range(k + 1, 16) if l >= 4], 0)
    assert np.isclose(f[-4], 4 / 16) and np.isclose(f[-3], np.log2(n) / 32)
    # above 65,536 rows the features see every ceil(n / 65,536)-th row: for
    # n = 200,001 that is every 4th row, 50,001 rows, and the size feature
    # is that sample's log2 / 32
    big = np.tile(P, (63, 1))[:200_001]
    fb = mlp.features(big)
    assert np.isclose(fb[-3], np.log2(50_001) / 32)
    # dimension 0 of row i is (i mod 32 + 0.5) / 32: every 4th row leaves 8
    # distinct values, 6,251 rows of residue 0 and 6,250 of each other one
    h0 = fb[:mlp.DMAX * mlp.BINS].reshape(16, 32)[0]
    assert np.count_nonzero(h0) == 8 and np.isclose(h0.sum(), 1.0)
    assert np.isclose(h0.max(), 6251 / 50_001) and np.isclose(h0[h0 > 0].min(), 6250 / 50_001)
    # a constant dimension has an empty correlation row
    Q = P.copy()
    Q[:, 1] = 0.3
    g = mlp.features(Q)
    assert g[mlp.DMAX * mlp.BINS + idx[(0, 1)]] == 0.0
    assert np.isclose(g[:mlp.DMAX * mlp.BINS].reshape(16, 32)[1, 0], 1.0)   # all in bin 0
