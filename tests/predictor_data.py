"""Training and evaluation data for the learned (Lambda_max, L) predictor,
and an FP64 restatement of its features for the parity test.

Matrices: m, n in [16, 128] with min(m, n) <= 64 (the batched path), rank 1-8
Gaussian product plus N(0, s^2) noise, s in [0.01, 0.2]; the response is
soft, hard or weighted soft (one third each) with a level f in [0.5, 3]
times the noise edge s (sqrt(m) + sqrt(n)) (weighted soft: c chosen so that
the weight near the noise edge is of that size, noise = max(m, n) s^2).

Labels come from the FP64 oracle.  Lambda_max is the 20-step power bound
(the one the learned path serves with); L* is the smallest L in [4, 96]
from which on every L' <= 96 gives a CPA within TOL = 1e-2 (relative
Frobenius) of the exact shrinkage, or 128 when there is none.  Tighter
targets are out of reach of 96 terms for most soft-threshold matrices of
this mix: the kink of the response limits the series' convergence.  The
error of the FP64 CPA is evaluated exactly from the singular values
(X H_hat(X^T X) and the exact shrinkage share singular vectors).  Targets:
t0 = log(sigma_max^2 / theta_4), t1 = log L*.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os

import numpy as np

import oracle as O

TOL = 1e-2
L_LO, L_HI, L_NONE = 4, 96, 128
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


def spectral_errors(sv, spec, lam, Ls):
    """Relative Frobenius error of the FP64 CPA for each L in Ls: the
    difference has singular values sigma_i |h_hat(sigma_i^2) - h(sigma_i^2)|
    with h_hat the shifted series on [0, lam] (oracle coefficients)."""
    sv = np.asarray(sv, dtype=np.float64)
    x = sv * sv
    hx = np.array([O.h(spec, v) for v in x])
    exact = float(np.sqrt(np.sum((sv * hx) ** 2)))
    denom = exact if exact > 0 else float(np.sqrt(np.sum(x)))
    xs = 2.0 * x / lam - 1.0
    out = []
    for L in Ls:
        c = O.coeffs(spec, L, lam).copy()
        c[0] *= 0.5
        hh = np.polynomial.chebyshev.chebval(xs, c)
        out.append(float(np.sqrt(np.sum((sv * (hh - hx)) ** 2))) / denom)
    return np.array(out)


def label(X32, spec):
    X = X32.astype(np.float64)
    m, n = X.shape
    p = min(m, n)
    tall = X if m >= n else X.T
    _, _, sv = O.svd_jacobi(tall)
    smax2 = float(np.max(sv)) ** 2
    v0 = O.start_vector(START_SEED, p)
    lam = O.lambda_bound(X, POWER_ITERS, MARGIN, v0)["lam"]
    th4 = O.lambda_bound(X, 3, MARGIN, v0)["theta"]
    Ls = np.arange(L_LO, L_HI + 1)
    ok = spectral_errors(sv, spec, lam, Ls) <= TOL
    Lstar = L_NONE
    for i in range(len(Ls) - 1, -1, -1):   # longest run of passing L ending at L_HI
        if not ok[i]:
            break
        Lstar = int(Ls[i])
    return math.log(smax2 / max(th4, 1e-300)), math.log(Lstar), sv


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


def _label_job(a):
    X, spec = a
    t0, t1, _ = label(X, spec)
    return t0, t1


def _exact_job(a):
    X, spec = a
    return O.shrink_exact(X.astype(np.float64), spec)


def _pool_map(fn, items):
    # spawn: a forked child of a process that has used the GPU can hang
    n = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(fn, items, chunksize=max(1, len(items) // (4 * n)))


def label_many(mats, specs):
    """(t0, t1) for every matrix, oracle-labelled in a process pool."""
    return np.array(_pool_map(_label_job, list(zip(mats, specs))))


def exact_many(mats, specs):
    """The oracle's exact shrinkage (Jacobi SVD) of every matrix."""
    return _pool_map(_exact_job, list(zip(mats, specs)))


def pack(mats):
    return np.concatenate([m.ravel() for m in mats]).astype(np.float32)
