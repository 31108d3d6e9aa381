"""Seeded synthetic workloads shaped like the paper's experiments.

This module is shared by the tests, the benchmark, the oracle checks and the
CUDA path's callers.  It holds no arithmetic of the shrinkage method itself:
only random matrices and the threshold parameters the workloads are quoted
with.  Every array is generated on the host with numpy's PCG64 so that the
oracle and the GPU see identical bits (returned as float32, the product's
input type; the oracle widens them to float64 exactly).

Workloads (the paper's own data, the Bricks/Office-windows images and the
Laboratory video of Section V, are not available; these stand in for them):

* ``single_lowrank``   256 x 256 rank-10 Gaussian product + N(0, 0.1^2) noise,
                       soft threshold at half the noise-spectrum edge.
* ``rpca_frame``       1024 x 1024 D = L0 + S0, L0 rank 30 with unit-norm
                       Gaussian factor columns, S0 5 % entries +-U[5,10]
                       (the background-modelling problem of Section V, Background Modeling of Video);
                       soft threshold tau = 1/mu, mu = mn / (4 |D|_1).
* ``patch_groups``     many 64 x c matrices, c uniform in [40, 80], rank-4
                       Gaussian signal + N(0, 0.05^2): patch groups of 8 x 8
                       patches with weighted soft thresholding.
* ``video_background`` 4096 x 8192: rank-5 Gaussian background, 3 % sparse
                       foreground +-U[0.5, 1], N(0, 0.01^2) noise.
* ``block_completion`` the synthetic matrix of Section V, Comparison with Existing Methods, J - blkdiag(0.5 1 1^T, n)
                       (rank n, entries 0.5 and 1) with a random x % of its
                       entries set to zero and marked unobserved.
* ``served_mix``       the learned predictor's serving mix: half patch-group
                       shapes (64 x U{40..80}), half sides log-uniform in
                       [64, 2048]; rank-r signal (unit-norm Gaussian factor
                       columns, singular values g_i times the noise edge
                       s (sqrt m + sqrt n), g_i log-uniform in [1.5, 40]) plus
                       N(0, s^2), s log-uniform in [0.01, 0.2]; hard, soft or
                       weighted soft thresholding (a third each) at f times
                       the noise edge, f uniform in [1.2, 3].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 170507112

HARD, SOFT, WSOFT = 0, 1, 2


@dataclass
class ShrinkSpec:
    kind: int = SOFT
    tau: float = 0.0
    c: float = 0.0
    eps: float = 1e-8
    noise: float = 0.0


@dataclass
class Workload:
    name: str
    X: np.ndarray                     # float32, m x n, row-major
    shrink: ShrinkSpec
    L: int                            # number of Chebyshev terms (alpha)
    power_iters: int = 20
    meta: dict = field(default_factory=dict)


def rng_for(config: int, index: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + 1000 * config + index)


def lowrank_gaussian(rng, m, n, rank, unit_columns=False):
    A = rng.standard_normal((m, rank))
    B = rng.standard_normal((n, rank))
    if unit_columns:
        A /= np.linalg.norm(A, axis=0, keepdims=True)
        B /= np.linalg.norm(B, axis=0, keepdims=True)
    return A @ B.T


def sparse_pm_uniform(rng, m, n, frac, lo, hi):
    S = np.zeros((m, n))
    mask = rng.random((m, n)) < frac
    k = int(mask.sum())
    mag = rng.uniform(lo, hi, size=k)
    sgn = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    S[mask] = sgn * mag
    return S


def noise_edge(m, n, sigma):
    """Largest singular value of an m x n N(0, sigma^2) matrix, to first order."""
    return sigma * (math.sqrt(m) + math.sqrt(n))


def single_lowrank(seed_index=0, m=256, n=256, rank=10, sigma=0.1, L=20) -> Workload:
    rng = rng_for(1, seed_index)
    X = lowrank_gaussian(rng, m, n, rank) + sigma * rng.standard_normal((m, n))
    tau = 0.5 * noise_edge(m, n, sigma)
    return Workload("single_lowrank_%dx%d_L%d" % (m, n, L), X.astype(np.float32),
                    ShrinkSpec(SOFT, tau), L, 20, {"rank": rank, "sigma": sigma})


def rpca_frame(seed_index=0, m=1024, n=1024, rank=30, frac=0.05, L=30) -> Workload:
    rng = rng_for(2, seed_index)
    L0 = lowrank_gaussian(rng, m, n, rank, unit_columns=True)
    S0 = sparse_pm_uniform(rng, m, n, frac, 5.0, 10.0)
    D = L0 + S0
    mu = m * n / (4.0 * np.abs(D).sum())
    return Workload("rpca_frame_%dx%d_L%d" % (m, n, L), D.astype(np.float32),
                    ShrinkSpec(SOFT, 1.0 / mu), L, 20,
                    {"mu": mu, "eta": 1.0 / math.sqrt(max(m, n)), "L0": L0.astype(np.float32),
                     "S0": S0.astype(np.float32)})


def patch_group_shapes(count, seed_index=0, m=64, cmin=40, cmax=80):
    rng = rng_for(3, 10_000_000 + seed_index)
    return [(m, int(c)) for c in rng.integers(cmin, cmax + 1, size=count)]


def patch_groups(count, seed_index=0, m=64, cmin=40, cmax=80, rank=4, sigma=0.05,
                 c_w=0.3, L=24):
    """Uneven patch-group matrices with the weighted-soft response.

    The noise energy subtracted in the weight's signal estimate is
    max(m, n) sigma^2 (the expected squared singular value of the noise
    block for the larger dimension)."""
    shapes = patch_group_shapes(count, seed_index, m, cmin, cmax)
    mats = []
    for i, (mm, nn) in enumerate(shapes):
        rng = rng_for(3, seed_index * 1_000_003 + i)
        X = lowrank_gaussian(rng, mm, nn, rank) + sigma * rng.standard_normal((mm, nn))
        mats.append(X.astype(np.float32))
    spec = ShrinkSpec(WSOFT, 0.0, c_w, 1e-8, 0.0)
    return mats, spec, L, sigma


def patch_group_noise(shape, sigma):
    return max(shape) * sigma * sigma


def video_background(seed_index=0, m=4096, n=8192, rank=5, frac=0.03, sigma=0.01, L=50,
                     kind=SOFT) -> Workload:
    rng = rng_for(4, seed_index)
    X = lowrank_gaussian(rng, m, n, rank)
    X += sparse_pm_uniform(rng, m, n, frac, 0.5, 1.0)
    X += sigma * rng.standard_normal((m, n))
    # noise level of the non-background part: N(0, sigma^2) plus the sparse
    # foreground's second moment frac * E[u^2], E[u^2] = 7/12 for u ~ U[0.5, 1]
    sig_hat = math.sqrt(sigma * sigma + frac * 7.0 / 12.0) * (math.sqrt(m) + math.sqrt(n))
    tau = 1.5 * sig_hat
    return Workload("video_background_%dx%d_L%d" % (m, n, L), X.astype(np.float32),
                    ShrinkSpec(kind, tau), L, 20, {"sig_hat": sig_hat})


def smooth_video(seed_index=0, side=16, frames=96, rank=3, frac=0.03, sigma=0.01):
    """Background-modelling frames whose background is smooth in space and
    time, so that a DCT over the frame index concentrates the frames' Gram
    matrix: D (side^2 pixels x frames) = sum_r A_r F_r^T + sparse +-U[0.5,1]
    foreground on frac of the entries + N(0, sigma^2), with A_r low-frequency
    2-D cosines over the frame (frequencies 0..2 per axis) and F_r
    low-frequency cosines over time (frequencies 0..2), random amplitudes."""
    rng = rng_for(6, seed_index)
    y, x = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5, indexing="ij")
    t = np.arange(frames) + 0.5
    D = np.zeros((side * side, frames))
    for _ in range(rank):
        a, b, c = rng.integers(0, 3, size=3)
        A = np.cos(np.pi * a * x / side) * np.cos(np.pi * b * y / side)
        F = np.cos(np.pi * c * t / frames)
        D += rng.uniform(0.5, 1.5) * np.outer(A.ravel(), F)
    D += sparse_pm_uniform(rng, side * side, frames, frac, 0.5, 1.0)
    D += sigma * rng.standard_normal(D.shape)
    m, n = D.shape
    mu = m * n / (4.0 * np.abs(D).sum())
    return D.astype(np.float32), mu, 1.0 / math.sqrt(max(m, n))


def random_gaussian(rng, m, n, scale=1.0):
    return (scale * rng.standard_normal((m, n))).astype(np.float32)


def block_completion(seed_index=0, size=1000, rank=100, frac_zero=0.10):
    """The synthetic completion input of Section V, Comparison with Existing Methods: D = J - blkdiag(D_s, rank)
    with J the all-ones size x size matrix and D_s = 0.5 * ones(b, b),
    b = size / rank (size a multiple of rank); a uniformly random set of
    round(frac_zero * size^2) entries is set to zero.  Returns (D, I, mask):
    the clean matrix, the corrupted one and the observation mask (uint8, 1 =
    observed, 0 = zeroed), all row-major."""
    if size % rank:
        raise ValueError("size must be a multiple of rank")
    b = size // rank
    blk = (np.arange(size)[:, None] // b) == (np.arange(size)[None, :] // b)
    D = np.where(blk, 0.5, 1.0)
    rng = rng_for(6, seed_index)
    nz = int(round(frac_zero * size * size))
    idx = rng.choice(size * size, size=nz, replace=False)
    mask = np.ones(size * size, dtype=np.uint8)
    mask[idx] = 0
    mask = mask.reshape(size, size)
    I = np.where(mask == 1, D, 0.0)
    return D.astype(np.float32), I.astype(np.float32), mask


# ---------------------------------------------------------------------------
# The learned predictor's serving mix (mixed sizes and kinds)

SERVED_CONFIG = 5


@dataclass
class ServedMatrix:
    X: np.ndarray          # float32 m x n
    shrink: ShrinkSpec
    family: int            # 0: patch-group shape, 1: log-uniform sides
    rank: int
    sigma: float           # noise standard deviation


def served_matrix(rng: np.random.Generator, family: int) -> ServedMatrix:
    """One matrix of the serving mix (recipe in the module docstring)."""
    if family == 0:
        m, n = 64, int(rng.integers(40, 81))
        r = int(rng.integers(1, 9))
    else:
        lo, hi = math.log(64.0), math.log(2048.0)
        m = int(round(math.exp(rng.uniform(lo, hi))))
        n = int(round(math.exp(rng.uniform(lo, hi))))
        r = int(rng.integers(1, min(50, min(m, n) // 4) + 1))
    s = float(math.exp(rng.uniform(math.log(0.01), math.log(0.2))))
    edge = s * (math.sqrt(m) + math.sqrt(n))
    g = np.sort(np.exp(rng.uniform(math.log(1.5), math.log(40.0), size=r)))[::-1]
    A = rng.standard_normal((m, r))
    A /= np.linalg.norm(A, axis=0)
    B = rng.standard_normal((r, n))
    B /= np.linalg.norm(B, axis=1)[:, None]
    X = (A * (g * edge)) @ B + s * rng.standard_normal((m, n))
    f = float(rng.uniform(1.2, 3.0))
    kind = int(rng.integers(0, 3))
    if kind == 0:
        spec = ShrinkSpec(HARD, f * edge)
    elif kind == 1:
        spec = ShrinkSpec(SOFT, f * edge)
    else:
        noise = max(m, n) * s * s
        c = f * edge * s * math.sqrt(min(m, n) + 2.0 * math.sqrt(m * n))
        spec = ShrinkSpec(WSOFT, 0.0, c, 1e-8, noise)
    return ServedMatrix(X.astype(np.float32), spec, family, r, s)


def served_one(seed_index: int, i: int, patch_fraction: float = 0.5) -> ServedMatrix:
    """Matrix i of the serving mix of seed_index; each matrix has its own
    generator, so any one can be regenerated alone."""
    rng = rng_for(SERVED_CONFIG, seed_index * 1000003 + i)
    family = 0 if rng.random() < patch_fraction else 1
    return served_matrix(rng, family)


def served_mix(count: int, seed_index: int = 0, patch_fraction: float = 0.5) -> list:
    """`count` matrices of the serving mix, seeded by seed_index."""
    return [served_one(seed_index, i, patch_fraction) for i in range(count)]
