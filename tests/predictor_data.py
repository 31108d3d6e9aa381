"""Patch-sized matrices for the batched kernel's predictor tests, and an
FP64 restatement of the predictor's twelve features for their parity tests.

Matrices: m, n in [16, 128] with min(m, n) <= 64 (the batched path), rank 1-8
Gaussian product plus N(0, s^2) noise, s in [0.01, 0.2]; the response is
soft, hard or weighted soft (one third each) with a level f in [0.5, 3]
times the noise edge s (sqrt(m) + sqrt(n)) (weighted soft: c chosen so that
the weight near the noise edge is of that size, noise = max(m, n) s^2).
The predictor's training labels (at the 1e-3 target, on the serving mix of
paper_1705_07112_gb300.inputs) are written by tests/golden/make_predictor_labels.py.
"""
from __future__ import annotations

import math
import numpy as np

import oracle as O

START_SEED = 0x1705071120000000
EDGE_SEED = START_SEED ^ 0x5EED
POWER_ITERS, MARGIN = 20, 0.01


def _shrink_for(rng, m, n, s):
    edge = s * (math.sqrt(m) + math.sqrt(n))
    f = float(rng.uniform(0.5, 3.0))
    kind = int(rng.integers(0, 3))
    if kind == 0:
        return O.Shrink(O.SOFT, f * edge)
    if kind == 1:
        return O.Shrink(O.HARD, f * edge)
    noise = max(m, n) * s * s
    c = f * edge * s * math.sqrt(min(m, n) + 2.0 * math.sqrt(m * n))
    return O.Shrink(O.WSOFT, 0.0, c, 1e-8, noise)


def generate(count, seed):
    rng = np.random.default_rng(seed)
    mats, specs = [], []
    while len(mats) < count:
        m, n = int(rng.integers(16, 129)), int(rng.integers(16, 129))
        if min(m, n) > 64:
            continue
        r = int(rng.integers(1, 9))
        s = float(np.exp(rng.uniform(math.log(0.01), math.log(0.2))))
        X = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + s * rng.standard_normal((m, n))
        mats.append(X.astype(np.float32))
        specs.append(_shrink_for(rng, m, n, s))
    return mats, specs


def reference_features(X32, spec):
    """The 12 features of cpa_batch_features in FP64 (oracle power steps)."""
    X = X32.astype(np.float64)
    m, n = X.shape
    p, q = min(m, n), max(m, n)
    G = X.T @ X if m >= n else X @ X.T
    v0 = O.start_vector(START_SEED, p)
    b4 = O.lambda_bound(X, 3, MARGIN, v0)
    th4, r4 = b4["theta"], b4["resid"]
    th2 = O.lambda_bound(X, 1, MARGIN, v0)["theta"]
    E = float(np.trace(G))
    E = E if E > 0 else 1.0
    tiny = 1e-30
    t4 = max(th4, tiny * E)
    u = O.start_vector(EDGE_SEED, p)
    for _ in range(4):
        u = th4 * u - G @ u
        u = u / np.linalg.norm(u)
    lmin = float(u @ G @ u) / float(u @ u)
    if spec.kind == O.WSOFT:
        w = spec.c / (math.sqrt(max(th4 - spec.noise, 0.0)) + spec.eps)
        thr2 = w * w
    else:
        thr2 = spec.tau ** 2
    thr2 = max(thr2, tiny * E)
    lm = max(lmin, tiny * E)
    fro = max(float(np.sum(G * G)), tiny * E * E)
    return np.array([
        math.log(p), math.log(q / p), math.log(E / t4), math.log(thr2 / t4),
        math.log(lm / t4), math.log(thr2 / lm), math.log(fro / (t4 * t4)),
        math.log(E / (p * thr2)), math.log(t4 / max(th2, tiny * E)), math.log((t4 + r4) / t4),
        1.0 if spec.kind == O.HARD else 0.0, 1.0 if spec.kind == O.WSOFT else 0.0,
    ])


def pack(mats):
    return np.concatenate([m.ravel() for m in mats]).astype(np.float32)
