"""Trains the learned (Lambda_max, L) predictor on the GPU and writes the
weights the learned shrinkage serves with.

Inputs: a labels file (targets per matrix of the serving mix, computed by
an exact reference: t0 = log(sigma_max^2 / theta_4), t1 = log L*, L* the
smallest order whose shrinkage is within the target error of the exact
one; see the file's own fields) and the seeded serving-mix generator of
this package, which regenerates every matrix from the file's seed index.

Steps, all on the GPU through the library:
  features   cpa_learn_features per matrix (12 features, theta_4);
  training   the 12 -> 64 -> 64 -> 2 network (cpa_mlp), standardised
             inputs, squared loss, AdamW steps (cpa_mlp_train_step) on
             random minibatches, learning rate decayed in steps;
  serving    the input standardisation folded into the first layer; the
             order scale L_scale from a quantile of the training residual
             of log L*; the bound margin from a quantile of the residual of
             t0 and the bound's floor, so the served bound covers
             sigma_max^2 for that quantile of the training matrices.
Matrices whose L* is beyond the label ladder (no order reaches the target)
keep their label (log of the sentinel): the network learns to predict a
large order for them, which the serving rule turns into the fallback.

    python -m paper_1705_07112_gb300.train_predictor --labels LABELS.npz \
        --out paper_1705_07112_gb300/predictor_c5.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import _lib, inputs

FEATURES = 12


def features_of(h, seed_index: int, idx, checksums=None, batch: int = 256):
    """Features and theta_4 of matrices `idx` of the serving mix
    (regenerated here; checksums, when given, must match to FP32 rounding)."""
    import torch
    F = np.zeros((len(idx), FEATURES), dtype=np.float32)
    th = np.zeros(len(idx), dtype=np.float64)
    Fd = torch.empty((batch, FEATURES), dtype=torch.float32, device="cuda")
    Td = torch.empty(batch, dtype=torch.float64, device="cuda")
    for b0 in range(0, len(idx), batch):
        keep = []
        for k, i in enumerate(idx[b0:b0 + batch]):
            sm = inputs.served_one(seed_index, int(i))
            if checksums is not None:
                cs = float(np.sum(sm.X, dtype=np.float64))
                want = float(checksums[b0 + k])
                if abs(cs - want) > 1e-4 * max(1.0, abs(want)):
                    raise RuntimeError("matrix %d of seed %d regenerated differently (%r vs %r)" % (i, seed_index,
                                                                                                 cs, want))
            X = torch.from_numpy(sm.X).cuda()
            sp = sm.shrink
            _lib.cpa_learn_features(h, X, dict(kind=sp.kind, tau=sp.tau, c=sp.c, eps=sp.eps, noise=sp.noise),
                                    F=Fd[k], theta=Td[k:k + 1])
            keep.append(X)   # alive until the features are copied back
        n = len(keep)
        F[b0:b0 + n] = Fd[:n].cpu().numpy()
        th[b0:b0 + n] = Td[:n].cpu().numpy()
    return F, th


def train(F, T, steps=6000, batch=512, seed=5, lr0=2e-3):
    """Network trained on standardised features; returns (net, mu, sd)."""
    import torch
    mu = F.mean(axis=0).astype(np.float64)
    sd = F.std(axis=0).astype(np.float64) + 1e-6
    Fn = torch.from_numpy(((F - mu) / sd).astype(np.float32)).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    net = _lib.MLP((FEATURES, 64, 64, 2), seed=seed)
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = len(F)
    for step in range(steps):
        ix = torch.randint(0, n, (batch,), device="cuda", generator=g)
        lr = lr0 if step < steps // 2 else (lr0 / 4 if step < 3 * steps // 4 else lr0 / 16)
        net.train_step(Fn[ix].contiguous(), Td[ix].contiguous(), lr, weight_decay=1e-5)
    return net, mu, sd


def fold_standardisation(net, mu, sd):
    """W1 x_n + b1 with x_n = (x - mu) / sd  ==  (W1 / sd) x + (b1 - (W1 / sd) mu)."""
    P = net.get_params().astype(np.float64)
    W1 = P[:FEATURES * 64].reshape(64, FEATURES)
    b1 = P[FEATURES * 64:FEATURES * 64 + 64]
    W1n = W1 / sd
    P[:FEATURES * 64] = W1n.ravel()
    P[FEATURES * 64:FEATURES * 64 + 64] = b1 - W1n @ mu
    net.set_params(P.astype(np.float32))
    return net


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--labels", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--order-quantile", type=float, default=0.85)
    ap.add_argument("--bound-quantile", type=float, default=0.995)
    a = ap.parse_args()
    t0 = time.time()
    lab = np.load(a.labels)
    seed_index = int(lab["seed_index"])
    idx = lab["i"]
    T = np.stack([lab["t0"], lab["t1"]], axis=1)
    h = _lib.Handle(0)
    F, th = features_of(h, seed_index, idx, checksums=lab["checksum"])
    t_feat = time.time() - t0
    net, mu, sd = train(F, T, steps=a.steps)
    net = fold_standardisation(net, mu, sd)
    y = net.forward(torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    r0, r1 = T[:, 0] - y[:, 0], T[:, 1] - y[:, 1]
    reach = lab["Lstar"] < int(lab["L_none"])
    L_scale = float(math.exp(np.quantile(r1[reach], a.order_quantile)))
    # the served bound max(theta_4 exp(max(y0, 0)) (1 + margin),
    # (theta_4 + r_4)(1 + 0.01)) must reach sigma_max^2: the smallest margin
    # (on a grid) doing so for the bound quantile of the training matrices
    th4, r4, smax2 = lab["theta4"], lab["r4"], lab["smax2"]
    floor = (th4 + r4) * 1.01
    pred = th4 * np.exp(np.maximum(y[:, 0], 0.0))
    margin = 1.0
    for mg in np.arange(0.01, 1.0, 0.005):
        if np.mean(np.maximum(pred * (1.0 + mg), floor) >= smax2) >= a.bound_quantile:
            margin = float(mg)
            break
    meta = {"labels": os.path.basename(a.labels), "seed_index": seed_index, "count": int(len(idx)),
            "steps": a.steps, "rms_t0": float(np.sqrt(np.mean(r0 ** 2))),
            "rms_t1": float(np.sqrt(np.mean(r1[reach] ** 2))), "L_scale": L_scale, "margin": margin,
            "order_quantile": a.order_quantile, "bound_quantile": a.bound_quantile,
            "feature_seconds": t_feat, "total_seconds": time.time() - t0}
    np.savez(a.out, params=net.get_params(), L_scale=L_scale, margin=margin, meta=json.dumps(meta))
    print(json.dumps(meta))
    net.close()
    h.close()


def load_predictor(path=None):
    """The trained network (an MLP on the current device) and its serving
    parameters {L_scale, margin} from a weights file written by main()."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "predictor_c5.npz")
    d = np.load(path)
    net = _lib.MLP((FEATURES, 64, 64, 2), seed=1)
    net.set_params(d["params"].astype(np.float32))
    return net, {"L_scale": float(d["L_scale"]), "margin": float(d["margin"]),
                 "meta": json.loads(str(d["meta"]))}


if __name__ == "__main__":
    main()
