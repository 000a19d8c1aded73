"""The learned proposal's kernels against the numpy oracle (oracle/mlp.py),
and the learned path's result against the plain path.

Floating-point tolerances: the kernels accumulate in binary32 where the oracle uses float64 with the same
bfloat16-rounded weights. A dot product of K <= 636 terms of magnitude <= 1
then differs by at most about K * 2^-24 relative per layer, so outputs are
compared with rtol = atol = 2e-4, gradients (two more layers of products)
with rtol = 2e-3 and atol = 1e-5. Histogram bins are computed in binary32 on
both sides and must agree exactly; correlations within 1e-4. The skyline of
the learned path must equal the plain path's exactly.
"""
import numpy as np
import pytest

import oracle
import skydata
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09993_b300 as sky  # noqa: E402


def _params(seed, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, omlp.n_params()).astype(np.float32)


def test_features_match_oracle():
    cases = [skydata.generate("independent", 5000, 4, 1), skydata.generate("anticorrelated", 200000, 9, 2),
             skydata.copula(70000, 16, 3, 0.6)[0], skydata.copula(131072 * 2 + 3, 3, 4, -0.4)[0]]
    C = cases[0].copy()
    C[:, 2] = 0.25                                      # a constant dimension
    cases.append(C)
    for P in cases:
        f, r = sky.features(torch.from_numpy(P).cuda())
        f = f.cpu().numpy()
        want = omlp.features(P)
        nb = omlp.DMAX * omlp.BINS
        assert np.allclose(f[:nb], want[:nb], rtol=0, atol=1e-7)
        assert np.allclose(f[nb:nb + 120], want[nb:nb + 120], atol=1e-4)
        assert np.allclose(f[nb + 120:], want[nb + 120:], atol=1e-6)
        S = P[::omlp.sample_stride(P.shape[0])]
        assert np.array_equal(r.cpu().numpy()[:P.shape[1]], S.min(axis=0))
        assert np.array_equal(r.cpu().numpy()[16:16 + P.shape[1]], S.max(axis=0))


def test_bf16_copy_and_forward_match_oracle():
    master = torch.from_numpy(_params(0)).cuda()
    wb = torch.empty(sky.MLP_PARAMS, dtype=torch.int16, device="cuda")
    sky.mlp_round(master, wb)
    got_bits = wb.cpu().numpy().view(np.uint16)
    want = omlp.bf16_round(master.cpu().numpy())
    assert np.array_equal(got_bits, (want.view(np.uint32) >> 16).astype(np.uint16))
    theta = want.astype(np.float64)
    rng = np.random.default_rng(1)
    F = rng.random((7, omlp.F_IN)).astype(np.float32)
    out = sky.mlp_forward(wb, torch.from_numpy(F).cuda()).cpu().numpy()
    for i in range(7):
        y, _ = omlp.forward(F[i].astype(np.float64), theta)
        assert np.allclose(out[i], y, rtol=2e-4, atol=2e-4)


def _batch(rng, B):
    F = rng.random((B, omlp.F_IN)).astype(np.float32)
    d = rng.integers(2, 17, size=B).astype(np.int32)
    labels = np.array([int(rng.integers(0, min(8, 24 // int(x)))) for x in d], dtype=np.int32)
    T = rng.random((B, 256)).astype(np.float32)
    M = np.zeros((B, 256), dtype=np.float32)
    for i, di in enumerate(d):
        M[i].reshape(16, 16)[:, :di] = 1
    return F, d, labels, T, M


def test_backward_matches_oracle():
    rng = np.random.default_rng(2)
    master = torch.from_numpy(_params(3, 0.2)).cuda()
    wb = torch.empty(sky.MLP_PARAMS, dtype=torch.int16, device="cuda")
    sky.mlp_round(master, wb)
    theta = omlp.bf16_round(master.cpu().numpy()).astype(np.float64)
    F, d, labels, T, M = _batch(rng, 33)
    c = lambda a: torch.from_numpy(a).cuda()
    loss, grad = sky.mlp_backward(wb, c(F), c(d), c(labels), c(T), c(M), 0.5)
    L, G = omlp.batch_loss_grad(theta, F.astype(np.float64), d, labels, T, M, 0.5)
    assert np.isclose(loss.item(), L, rtol=1e-4)
    g = grad.cpu().numpy()
    assert np.allclose(g, G, rtol=2e-3, atol=1e-5)


def test_adamw_matches_oracle():
    rng = np.random.default_rng(4)
    master0 = _params(5)
    g = rng.normal(0, 1e-2, omlp.n_params()).astype(np.float32)
    master = torch.from_numpy(master0.copy()).cuda()
    wb = torch.empty(sky.MLP_PARAMS, dtype=torch.int16, device="cuda")
    m = torch.zeros(sky.MLP_PARAMS, device="cuda")
    v = torch.zeros(sky.MLP_PARAMS, device="cuda")
    th, mo, vo = master0.astype(np.float64), np.zeros(master0.size), np.zeros(master0.size)
    for step in (1, 2, 3):
        sky.mlp_adamw(master, wb, m, v, torch.from_numpy(g).cuda(), step, 1e-3, 1e-2)
        th, mo, vo = omlp.adamw(th, g.astype(np.float64), mo, vo, step, 1e-3, 1e-2)
    assert np.allclose(master.cpu().numpy(), th, rtol=1e-5, atol=1e-7)
    bits = wb.cpu().numpy().view(np.uint16)
    assert np.array_equal(bits, (omlp.bf16_round(master.cpu().numpy()).view(np.uint32) >> 16).astype(np.uint16))


def test_learned_path_result_equals_plain_path():
    wb = torch.empty(sky.MLP_PARAMS, dtype=torch.int16, device="cuda")
    for seed, (kind, n, d) in enumerate([("independent", 30000, 6), ("anticorrelated", 20000, 4),
                                         ("correlated", 50000, 10)]):
        sky.mlp_round(torch.from_numpy(_params(10 + seed, 0.3)).cuda(), wb)
        P = skydata.generate(kind, n, d, seed)
        x = torch.from_numpy(P).cuda()
        want = oracle.skyline_sfs(P).tolist()
        assert sky.skyline_learned(x, wb).cpu().tolist() == want
        lg, prop = sky.propose(x, wb)
        assert 1 <= lg <= 8 and lg * d <= 24 and tuple(prop.shape) == (16, d)


def test_training_steps_reduce_loss():
    rng = np.random.default_rng(6)
    master = torch.from_numpy(_params(7, 0.05)).cuda()
    wb = torch.empty(sky.MLP_PARAMS, dtype=torch.int16, device="cuda")
    sky.mlp_round(master, wb)
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    F, d, labels, T, M = _batch(rng, 64)
    c = lambda a: torch.from_numpy(a).cuda()
    F, d, labels, T, M = map(c, (F, d, labels, T, M))
    first = None
    for step in range(1, 61):
        loss, grad = sky.mlp_backward(wb, F, d, labels, T, M, 1.0)
        first = loss.item() if first is None else first
        sky.mlp_adamw(master, wb, m, v, grad, step, 3e-3, 0.0)
    assert loss.item() < 0.5 * first
