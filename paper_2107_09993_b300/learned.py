"""Training and evaluation of the learned proposal (host driver).

Every numerical step runs in libsky's CUDA kernels (features, forward,
backward, AdamW); this module only generates the synthetic training sets,
labels them with the plain skyline path, batches them and keeps checkpoints.

Labels, per training set (Gaussian copula, n = 100,000, d ~ U{2..16},
rho ~ U[-0.9, 0.9], seed 1000 + k):
* filter points: for 16 fixed positive weight vectors w_j, the skyline point
  (from the plain path) minimising w_j . x_hat, in the coordinates x_hat
  normalised by the sample's min / max. Such minimisers dominate a large
  share of the data in direction w_j.
* layer: the admissible grid layer log2_g (log2_g * d <= 24) with the lowest
  measured time of the skyline call with those 16 filter points (what the
  learned path runs), best of three runs; a layer within 3% of the best time
  loses to the automatic layer, so timing noise does not move the label away
  from the automatic policy.

At inference (sky_propose with n_ref = the training size) the predicted
layer is moved by the automatic policy's change from the training size to
the set's size, so the network only has to learn the correction that the
distribution calls for.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "learned_weights.npz")
N_FILT, DMAX, N_LAYERS = 16, 16, 8


def directions(seed: int = 7) -> np.ndarray:
    """16 fixed weight vectors over 16 dimensions (Dirichlet(1) draws)."""
    return np.random.default_rng(seed).dirichlet(np.ones(DMAX), size=N_FILT)


def auto_layer(n: int, d: int) -> int:
    """The plain path's automatic layer for n rows in d dimensions (the
    library's rule: the largest log2_g <= min(8, 24 / d) with
    2^(log2_g d) <= 32 n)."""
    r = max(1, min(8, 24 // d))
    while r > 1 and (1 << (r * d)) > 32.0 * max(n, 1):
        r -= 1
    return r


def admissible_layers(d: int):
    return [lg for lg in range(1, N_LAYERS + 1) if lg * d <= 24]


def _time_ms(fn, reps=2):
    import torch
    best = float("inf")
    out = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best, out


def label_set(x, W=None, reps=3, tie=1.03):
    """Features, layer label and filter targets of one device point set."""
    import torch
    import paper_2107_09993_b300 as sky

    if W is None:
        W = directions()
    n, d = x.shape
    feat, rng = sky.features(x)
    sky_idx = sky.skyline(x).long()
    lo = rng[:d]
    hi = rng[16:16 + d]
    span = torch.where(hi > lo, hi - lo, torch.ones_like(hi))
    S = (x[sky_idx] - lo) / span
    Wd = torch.from_numpy(W[:, :d] / W[:, :d].sum(axis=1, keepdims=True)).to(x.device, torch.float32)
    pick = torch.argmin(S @ Wd.T, dim=0)
    filt = x[sky_idx[pick]].contiguous()
    times = {}
    for lg in admissible_layers(d):
        times[lg] = _time_ms(lambda: sky.skyline(x, log2_g=lg, filter_points=filt), reps)[0]
    best = min(times, key=times.get)
    auto = auto_layer(n, d)
    if auto in times and times[auto] <= tie * times[best]:
        best = auto
    target = torch.zeros((N_FILT, DMAX), device=x.device)
    target[:, :d] = S[pick]
    mask = torch.zeros((N_FILT, DMAX), device=x.device)
    mask[:, :d] = 1.0
    return feat, best - 1, target.reshape(-1), mask.reshape(-1), times


def make_training_set(count=10000, n=100000, seed0=1000, path=None, log_every=500):
    """Generates and labels `count` copula sets; saves an .npz if `path`."""
    import torch
    import skydata

    rng = np.random.default_rng(seed0)
    W = directions()
    F = np.zeros((count, 636), np.float32)
    D = np.zeros(count, np.int32)
    L = np.zeros(count, np.int32)
    T = np.zeros((count, 256), np.float32)
    M = np.zeros((count, 256), np.float32)
    best_ms = np.zeros(count, np.float32)
    auto_ms = np.zeros(count, np.float32)
    layer_ms = np.full((count, N_LAYERS), np.nan, np.float32)
    t0 = time.time()
    for k in range(count):
        d = int(rng.integers(2, 17))
        rho = float(rng.uniform(-0.9, 0.9))
        x, _ = skydata.copula_torch(n, d, seed0 + k, rho)
        feat, lab, tgt, msk, times = label_set(x, W)
        F[k] = feat.cpu().numpy()
        D[k], L[k] = d, lab
        T[k] = tgt.cpu().numpy()
        M[k] = msk.cpu().numpy()
        best_ms[k] = min(times.values())
        for lg, ms in times.items():
            layer_ms[k, lg - 1] = ms
        import paper_2107_09993_b300 as sky
        auto_ms[k] = _time_ms(lambda: sky.skyline(x))[0]
        if log_every and (k + 1) % log_every == 0:
            print(f"[learned] labelled {k + 1}/{count} sets in {time.time() - t0:.1f}s", flush=True)
        del x
    data = dict(features=F, dims=D, labels=L, targets=T, masks=M, best_ms=best_ms, auto_ms=auto_ms,
                layer_ms=layer_ms)
    if path:
        np.savez_compressed(path, **data)
    return data


class Trainer:
    """AdamW training of the proposal network with libsky's kernels, with
    checkpoint / resume (weights, moments, step and the shuffling RNG)."""

    def __init__(self, seed=0, lr=1e-3, wd=1e-4, lam=1.0, batch=256, ckpt=None):
        import torch
        import paper_2107_09993_b300 as sky

        self.sky = sky
        self.lr, self.wd, self.lam, self.batch = lr, wd, lam, batch
        self.ckpt = ckpt
        self.rng = np.random.default_rng(seed)
        P = sky.MLP_PARAMS
        # He-style initialisation per layer
        w = []
        for (out, inp) in ((64, 636), (64, 64), (264, 64)):
            w.append(self.rng.normal(0, np.sqrt(2.0 / inp), out * inp))
            w.append(np.zeros(out))
        self.master = torch.from_numpy(np.concatenate(w).astype(np.float32)).cuda()
        assert self.master.numel() == P
        self.wb = torch.empty(P, dtype=torch.int16, device="cuda")
        sky.mlp_round(self.master, self.wb)
        self.m = torch.zeros(P, device="cuda")
        self.v = torch.zeros(P, device="cuda")
        self.step = 0
        if ckpt and os.path.exists(ckpt):
            self.load(ckpt)

    def save(self, path):
        np.savez(path, master=self.master.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 step=self.step, rng=json.dumps(self.rng.bit_generator.state))

    def load(self, path):
        import torch
        z = np.load(path, allow_pickle=False)
        self.master.copy_(torch.from_numpy(z["master"]))
        self.m.copy_(torch.from_numpy(z["m"]))
        self.v.copy_(torch.from_numpy(z["v"]))
        self.step = int(z["step"])
        self.rng.bit_generator.state = json.loads(str(z["rng"]))
        self.sky.mlp_round(self.master, self.wb)

    def fit(self, data, epochs=40, ckpt_every=200, log=True):
        import torch
        dev = "cuda"
        F = torch.from_numpy(data["features"]).to(dev)
        D = torch.from_numpy(data["dims"]).to(dev)
        L = torch.from_numpy(data["labels"]).to(dev)
        T = torch.from_numpy(data["targets"]).to(dev)
        M = torch.from_numpy(data["masks"]).to(dev)
        N = F.shape[0]
        history = []
        for ep in range(epochs):
            perm = torch.from_numpy(self.rng.permutation(N)).to(dev)
            tot, nb = 0.0, 0
            for b0 in range(0, N - self.batch + 1, self.batch):
                idx = perm[b0:b0 + self.batch]
                loss, grad = self.sky.mlp_backward(self.wb, F[idx].contiguous(), D[idx].contiguous(),
                                                   L[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous(),
                                                   self.lam)
                self.step += 1
                self.sky.mlp_adamw(self.master, self.wb, self.m, self.v, grad, self.step, self.lr, self.wd)
                tot += loss.item()
                nb += 1
                if self.ckpt and self.step % ckpt_every == 0:
                    self.save(self.ckpt)
            history.append(tot / max(nb, 1))
            if log:
                print(f"[learned] epoch {ep + 1}/{epochs} loss {history[-1]:.4f}", flush=True)
        return history

    def accuracy(self, data):
        import torch
        out = self.sky.mlp_forward(self.wb, torch.from_numpy(data["features"]).cuda()).cpu().numpy()
        pred = []
        for i, d in enumerate(data["dims"]):
            ok = [c for c in range(N_LAYERS) if (c + 1) * int(d) <= 24]
            pred.append(max(ok, key=lambda c: out[i, c]))
        pred = np.array(pred)
        return float((pred == data["labels"]).mean()), pred

    def export(self, path=WEIGHTS, meta=None):
        bits = self.wb.cpu().numpy().view(np.uint16)
        np.savez(path, bf16=bits, meta=json.dumps(meta or {}))


def load_weights(path=WEIGHTS, device="cuda"):
    """Trained bfloat16 parameters as an int16 CUDA tensor (bit pattern)."""
    import torch
    z = np.load(path, allow_pickle=False)
    return torch.from_numpy(z["bf16"].view(np.int16).copy()).to(device), json.loads(str(z["meta"]))


def evaluate_sets(params, sets, reps=3, n_ref=None):
    """Plain (automatic layer, no proposals) versus learned path on device
    point sets: best-of-`reps` times and a check that both return the same
    indices. `sets` is a list of (name, tensor)."""
    import torch
    import paper_2107_09993_b300 as sky

    n_ref = sky.TRAIN_ROWS if n_ref is None else n_ref
    rows = []
    for name, x in sets:
        t_plain, a = _time_ms(lambda: sky.skyline(x), reps)
        st_plain = sky.last_run_stats()
        t_prop, _ = _time_ms(lambda: sky.propose(x, params, n_ref=n_ref), reps)
        t_learn, b = _time_ms(lambda: sky.skyline_learned(x, params, n_ref=n_ref), reps)
        st_learn = sky.last_run_stats()
        rows.append({"set": name, "n": int(x.shape[0]), "d": int(x.shape[1]), "plain_ms": round(t_plain, 3),
                     "learned_ms": round(t_learn, 3), "propose_ms": round(t_prop, 3),
                     "speedup": round(t_plain / t_learn, 3),
                     "identical": bool(torch.equal(a, b)), "skyline": int(a.numel()),
                     "plain_layer": st_plain["log2_g"], "learned_layer": st_learn["log2_g"],
                     "survivors_plain": st_plain["survivors"], "survivors_learned": st_learn["survivors"],
                     "filters_used": st_learn["n_filter_used"]})
    return rows


def main(argv=None):
    import argparse
    import torch
    import skydata

    ap = argparse.ArgumentParser(description="train / evaluate the learned proposal on the GPU")
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--count", type=int, default=10000)
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--data", default=None, help="cache of the labelled sets (.npz)")
    ap.add_argument("--ckpt", default=None)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--eval-n", type=int, default=10_000_000)
    args = ap.parse_args(argv)
    if args.cmd == "train":
        t0 = time.time()
        if args.data and os.path.exists(args.data):
            data = dict(np.load(args.data))
        else:
            data = make_training_set(args.count, args.n, path=args.data)
        t_label = time.time() - t0
        N = data["features"].shape[0]
        split = int(N * 0.9)
        train = {k: v[:split] for k, v in data.items()}
        held = {k: v[split:] for k, v in data.items()}
        tr = Trainer(ckpt=args.ckpt)
        hist = tr.fit(train, epochs=args.epochs)
        acc, pred = tr.accuracy(held)
        # on held-out sets: time of the predicted layer and of the automatic
        # layer (both with the target filter points) over the best layer's
        regret = {}
        if "layer_ms" in held:
            lm = held["layer_ms"]
            rows = np.arange(lm.shape[0])
            best = np.nanmin(lm, axis=1)
            # the automatic layer is above the network's range (8) for d <= 2
            auto = np.array([auto_layer(args.n, int(d)) - 1 for d in held["dims"]])
            inr = auto < N_LAYERS
            regret = {"held_out_pred_over_best": float(np.mean(lm[rows, pred] / best)),
                      "held_out_pred_over_best_d3plus": float(np.mean((lm[rows, pred] / best)[inr])),
                      "held_out_auto_over_best_d3plus": float(np.mean(lm[rows[inr], auto[inr]] / best[inr]))}
        meta = {"sets": N, "rows_per_set": args.n, "train_sets": split, "held_out": N - split, "epochs": args.epochs,
                "final_loss": hist[-1], "held_out_layer_accuracy": acc, "label_seconds": round(t_label, 1),
                "steps": tr.step, **regret}
        tr.export(args.out, meta)
        print(json.dumps(meta), flush=True)
    else:
        params, meta = load_weights(args.out)
        sets = []
        for rho in (-0.8, 0.0, 0.8):
            P, _ = skydata.copula(args.eval_n, 8, 3, rho)
            sets.append((f"copula rho={rho}", torch.from_numpy(P).cuda()))
        for row in evaluate_sets(params, sets, n_ref=int(meta.get("rows_per_set", args.n))):
            print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
