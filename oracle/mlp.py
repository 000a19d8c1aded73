"""Oracle of the learned proposal -- test infrastructure only (see __init__).

Plain numpy, float64 unless a step is defined in binary32. It mirrors what
the CUDA kernels compute, written from the definitions:

* features(P): per-dimension 32-bin histograms of the min/max-normalised
  values and the Pearson correlation of every pair of dimensions, over a
  strided row sample of s rows, plus (d/16, log2(s)/32). Normalised value and bin are
  binary32 expressions, so the bins are exact; correlations are float64.
* forward / backward: a 3-layer perceptron 636 -> 64 -> 64 -> 264 with ReLU,
  weights rounded to bfloat16 (round to nearest even), float64 arithmetic.
* loss: cross-entropy over the admissible grid layers (log2_g * d <= 24)
  plus lambda times the masked mean squared error of the 16 filter points.
* adamw: decoupled weight decay Adam.
"""
from __future__ import annotations

import numpy as np

DMAX = 16
BINS = 32
N_LAYERS = 8            # classes: log2_g = 1 .. 8
N_FILT = 16
F_IN = DMAX * BINS + DMAX * (DMAX - 1) // 2 + 4    # 636
HID = 64
OUT = N_LAYERS + N_FILT * DMAX                     # 264
SAMPLE = 65536
SHAPES = [(HID, F_IN), (HID,), (HID, HID), (HID,), (OUT, HID), (OUT,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unflatten(theta):
    out, at = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(theta[at:at + k], dtype=np.float64).reshape(s))
        at += k
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def sample_stride(n: int) -> int:
    return max(1, -(-n // SAMPLE))


def valid_layers(d: int) -> np.ndarray:
    """Mask of admissible classes: class c is log2_g = c + 1, needs log2_g*d <= 24."""
    return np.array([(c + 1) * d <= 24 for c in range(N_LAYERS)])


def features(P) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float32)
    n, d = P.shape
    S = P[::sample_stride(n)]
    s = S.shape[0]
    mn = S.min(axis=0)
    mx = S.max(axis=0)
    rng = (mx - mn).astype(np.float32)
    inv = np.where(rng > 0, np.float32(1.0) / np.where(rng > 0, rng, np.float32(1)), np.float32(0)).astype(np.float32)
    xh = ((S - mn).astype(np.float32) * inv).astype(np.float32)
    xh = np.clip(xh, np.float32(0), np.float32(1))
    b = np.minimum(np.floor(xh * np.float32(BINS)).astype(np.int64), BINS - 1)
    hist = np.zeros((DMAX, BINS))
    for k in range(d):
        hist[k] = np.bincount(b[:, k], minlength=BINS) / s
    X = xh.astype(np.float64)
    mu = X.mean(axis=0)
    C = (X - mu).T @ (X - mu) / s
    var = np.diag(C)
    corr = np.zeros((DMAX, DMAX))
    for k in range(d):
        for l in range(d):
            if var[k] > 0 and var[l] > 0:
                corr[k, l] = C[k, l] / np.sqrt(var[k] * var[l])
    tri = [corr[k, l] for k in range(DMAX) for l in range(k + 1, DMAX)]
    extra = [d / 16.0, np.log2(s) / 32.0, 0.0, 0.0]
    return np.concatenate([hist.ravel(), np.array(tri), np.array(extra)])


def forward(f, theta):
    W1, b1, W2, b2, W3, b3 = unflatten(theta)
    z1 = W1 @ f + b1
    h1 = np.maximum(z1, 0)
    z2 = W2 @ h1 + b2
    h2 = np.maximum(z2, 0)
    y = W3 @ h2 + b3
    return y, (f, h1, h2)


def loss(y, d, layer_label, target, mask, lam):
    """Returns (loss, dL/dy) for one sample."""
    v = valid_layers(d)
    z = np.where(v, y[:N_LAYERS], -np.inf)
    zmax = z[v].max()
    e = np.where(v, np.exp(z - zmax), 0.0)
    p = e / e.sum()
    ce = -np.log(p[layer_label])
    dy = np.zeros(OUT)
    dy[:N_LAYERS] = p
    dy[layer_label] -= 1.0
    cnt = max(mask.sum(), 1.0)
    r = (y[N_LAYERS:] - target) * mask
    mse = (r * r).sum() / cnt
    dy[N_LAYERS:] = lam * 2.0 * r / cnt
    return ce + lam * mse, dy


def backward(theta, cache, dy):
    W1, b1, W2, b2, W3, b3 = unflatten(theta)
    f, h1, h2 = cache
    gW3 = np.outer(dy, h2)
    gb3 = dy.copy()
    dh2 = (W3.T @ dy) * (h2 > 0)
    gW2 = np.outer(dh2, h1)
    gb2 = dh2
    dh1 = (W2.T @ dh2) * (h1 > 0)
    gW1 = np.outer(dh1, f)
    gb1 = dh1
    return flatten([gW1, gb1, gW2, gb2, gW3, gb3])


def batch_loss_grad(theta, F, d, labels, targets, masks, lam):
    """Mean loss and gradient over a batch."""
    L, G = 0.0, np.zeros(theta.size)
    B = F.shape[0]
    for i in range(B):
        y, cache = forward(F[i], theta)
        li, dy = loss(y, int(d[i]), int(labels[i]), targets[i], masks[i], lam)
        L += li / B
        G += backward(theta, cache, dy) / B
    return L, G


def adamw(theta, g, m, v, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
