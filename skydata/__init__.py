"""Seeded synthetic inputs for the skyline path and its oracle.

This module only draws numbers. It holds none of the skyline arithmetic
(no dominance test, no cell mapping), so the CUDA path and the CPU oracle can
both take their inputs from here without sharing any of the method.

Distribution families follow the paper's experimental section (Sec. 7.1:
Independent, Correlated, Anti-correlated), with the concrete recipes below
standing in for the original generator, which is not available:

* independent     x ~ U[0,1)^d, float32 drawn directly.
* correlated      t ~ U[0,1), x_k = clip(t + N(0, 0.05), 0, 1).
* anticorrelated  u ~ U[0,1)^d, c ~ N(0.5, 0.05) per point,
                  x = clip(u - mean(u) + c, 0, 1)  (sum x = d*c before clipping).
* copula          Gaussian copula with equicorrelation rho, clamped to be
                  positive definite (rho >= -0.95/(d-1)), u = Phi(z) < 1.
All values are produced in float64 by numpy's PCG64 stream and cast to float32,
except `independent`, which draws float32 directly.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "independent", "correlated", "anticorrelated", "copula", "generate",
    "mixed_table", "batched_queries", "GENERATORS", "generate_torch",
]


def independent(n: int, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random((n, d), dtype=np.float32)


def correlated(n: int, d: int, seed: int, sigma: float = 0.05) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = rng.random((n, 1))
    x = t + rng.normal(0.0, sigma, size=(n, d))
    return np.clip(x, 0.0, 1.0).astype(np.float32)


def anticorrelated(n: int, d: int, seed: int, sigma: float = 0.05) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 20  # bounded float64 temporaries for n = 1e7
    for s in range(0, n, step):
        m = min(step, n - s)
        u = rng.random((m, d))
        c = rng.normal(0.5, sigma, size=(m, 1))
        x = u - u.mean(axis=1, keepdims=True) + c
        out[s:s + m] = np.clip(x, 0.0, 1.0)
    return out


def copula(n: int, d: int, seed: int, rho: float) -> tuple[np.ndarray, float]:
    """Gaussian copula sample; returns (points, effective rho)."""
    from scipy.special import ndtr

    rng = np.random.default_rng(seed)
    rho_eff = float(rho)
    if d > 1:
        rho_eff = max(rho_eff, -0.95 / (d - 1))
    cov = np.full((d, d), rho_eff)
    np.fill_diagonal(cov, 1.0)
    chol = np.linalg.cholesky(cov)
    z = rng.standard_normal((n, d)) @ chol.T
    u = ndtr(z)
    u = np.minimum(u, np.nextafter(1.0, 0.0))
    x = u.astype(np.float32)
    x = np.minimum(x, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))))
    return x, rho_eff


GENERATORS = {
    "independent": independent,
    "correlated": correlated,
    "anticorrelated": anticorrelated,
}


def generate(kind: str, n: int, d: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(GENERATORS[kind](n, d, seed))


def mixed_table(n_rows: int, n_cols: int, seed: int) -> np.ndarray:
    """First half independent, second half anti-correlated (one float32 table)."""
    half = n_rows // 2
    t = np.empty((n_rows, n_cols), dtype=np.float32)
    t[:half] = independent(half, n_cols, seed)
    t[half:] = anticorrelated(n_rows - half, n_cols, seed + 1)
    return t


def batched_queries(n_queries: int, n_rows: int, n_cols: int, seed: int,
                    n_lo: float = 1e3, n_hi: float = 1e6,
                    d_lo: int = 2, d_hi: int = 12) -> np.ndarray:
    """Uneven subspace / row-range queries.

    Returns an int64 array [n_queries, 3] of (row_begin, row_count, dim_mask):
    row_count log-uniform in [n_lo, n_hi], d uniform in {d_lo..d_hi}, a random
    subset of d distinct columns, and a uniform valid start row.
    """
    rng = np.random.default_rng(seed)
    q = np.empty((n_queries, 3), dtype=np.int64)
    for i in range(n_queries):
        cnt = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        cnt = max(1, min(cnt, n_rows))
        dq = int(rng.integers(d_lo, min(d_hi, n_cols) + 1))
        dims = rng.choice(n_cols, size=dq, replace=False)
        mask = 0
        for k in dims:
            mask |= 1 << int(k)
        start = int(rng.integers(0, n_rows - cnt + 1))
        q[i] = (start, cnt, mask)
    return q


def copula_torch(n: int, d: int, seed: int, rho: float, device="cuda"):
    """Gaussian copula sample drawn on the GPU with torch (seeded), for the
    learned proposal's training sets: same recipe as `copula`, float32 in
    [0, 1). Returns (points tensor [n, d], effective rho)."""
    import torch

    rho_eff = float(rho)
    if d > 1:
        rho_eff = max(rho_eff, -0.95 / (d - 1))
    cov = torch.full((d, d), rho_eff, dtype=torch.float64)
    cov.fill_diagonal_(1.0)
    chol = torch.linalg.cholesky(cov).to(device=device, dtype=torch.float32)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    z = torch.randn((n, d), generator=g, device=device, dtype=torch.float32) @ chol.T
    u = 0.5 * torch.erfc(-z / math.sqrt(2.0))
    return torch.clamp(u, max=float(np.nextafter(np.float32(1.0), np.float32(0.0)))).contiguous(), rho_eff


def generate_torch(kind: str, n: int, d: int, seed: int, device="cuda", block: int = 1 << 26):
    """The three families drawn on the GPU with torch (float32 arithmetic,
    seeded per block of rows), for sets too large to draw on the host (the
    paper's 3.2e9-point runs). Same recipes as the numpy generators, not the
    same numbers. Returns a [n, d] float32 CUDA tensor."""
    import torch

    out = torch.empty((n, d), dtype=torch.float32, device=device)
    g = torch.Generator(device=device)
    for b, s in enumerate(range(0, n, block)):
        m = min(block, n - s)
        g.manual_seed(int(seed) * 1_000_003 + b)
        if kind == "independent":
            out[s:s + m] = torch.rand((m, d), generator=g, device=device)
        elif kind == "correlated":
            t = torch.rand((m, 1), generator=g, device=device)
            out[s:s + m] = (t + 0.05 * torch.randn((m, d), generator=g, device=device)).clamp_(0.0, 1.0)
        elif kind == "correlated_inside":
            # the correlated recipe with rows outside [0, 1)^d drawn again
            # instead of clipped (no pile of points on the faces of the cube)
            x = torch.rand((m, 1), generator=g, device=device) + 0.05 * torch.randn((m, d), generator=g, device=device)
            bad = ((x < 0) | (x >= 1)).any(dim=1)
            while bool(bad.any()):
                k = int(bad.sum())
                y = torch.rand((k, 1), generator=g, device=device) + 0.05 * torch.randn((k, d), generator=g,
                                                                                         device=device)
                x[bad] = y
                bad = ((x < 0) | (x >= 1)).any(dim=1)
            out[s:s + m] = x
        elif kind == "anticorrelated":
            u = torch.rand((m, d), generator=g, device=device)
            c = 0.5 + 0.05 * torch.randn((m, 1), generator=g, device=device)
            out[s:s + m] = (u - u.mean(dim=1, keepdim=True) + c).clamp_(0.0, 1.0)
        else:
            raise ValueError(kind)
    return out
