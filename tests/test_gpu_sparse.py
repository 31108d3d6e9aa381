"""The sparsity-based reduction on the device (transform, entry threshold,
X T^T H(Phi_) T) against the oracle's Algorithm 1 with the same T and eps,
with the recurrence on the full thresholded operand and on the block of its
nonzero rows (CPA_OPT_SPARSE_COMPACT), which the smooth inputs here make
small: the two routes compute the same filter.

T is built here from its definition (independently of the library's
generator); eps is chosen in a wide gap of the oracle's |Phi| values so that
the FP32 and FP64 sides keep the same entries.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module")
def cpa():
    import __graft_entry__ as g
    g.build()
    import paper_1705_07112_gb300 as cpa
    return cpa


@pytest.fixture(scope="module")
def handle(cpa):
    h = cpa.Handle(0)
    yield h
    h.close()


def dct(size):
    T = np.zeros((size, size))
    for k in range(size):
        s = math.sqrt((1.0 if k == 0 else 2.0) / size)
        for j in range(size):
            T[k, j] = s * math.cos(math.pi * (2 * j + 1) * k / (2 * size))
    return T


def transform(kind, p):
    if kind == 0:
        return np.eye(p)
    if kind == 1:
        T = np.zeros((p, p))
        for i in range(p // 2):
            T[i, 2 * i] = T[i, 2 * i + 1] = math.sqrt(0.5)
        if p % 2:
            T[p // 2, p - 1] = 1.0
        return T
    if kind == 2:
        T = np.zeros((p, p))
        for b in range(0, p, 8):
            sz = min(8, p - b)
            T[b:b + sz, b:b + sz] = dct(sz)
        return T
    return dct(p)


def gap_threshold(Phi, lo_frac=0.002, hi_frac=0.9):
    """eps in the widest multiplicative gap of |Phi| within a rank window,
    and the rank k of the smallest kept entry."""
    a = np.sort(np.abs(Phi).ravel())[::-1]
    n = a.size
    best, kbest = 0.0, None
    for k in range(max(1, int(lo_frac * n)), int(hi_frac * n)):
        if a[k] <= 0:
            if a[k - 1] > 0:   # the exact zeros of a block-structured Phi
                return 0.5 * a[k - 1], k, math.inf
            break
        r = a[k - 1] / a[k]
        if r > best:
            best, kbest = r, k
    eps = math.sqrt(a[kbest - 1] * a[kbest])
    return eps, kbest, best


def smooth_matrix(rng, m, n):
    # columns are smooth (low-frequency cosines) so the transforms sparsify
    t = np.linspace(0, 1, min(m, n) if m >= n else m)
    if m >= n:
        base = np.stack([np.cos(math.pi * f * np.linspace(0, 1, n)) for f in range(4)])
        X = rng.standard_normal((m, 4)) @ base + 0.01 * rng.standard_normal((m, n))
    else:
        base = np.stack([np.cos(math.pi * f * np.linspace(0, 1, m)) for f in range(4)]).T
        X = base @ rng.standard_normal((4, n)) + 0.01 * rng.standard_normal((m, n))
    return X.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [(120, 64), (64, 120), (90, 37), (37, 90)])
@pytest.mark.parametrize("tkind", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("compact", [1, 0])
def test_sparsify_matches_oracle(cpa, handle, shape, tkind, mode, prec, compact):
    import torch
    if tkind == 0 and mode == 0:
        pytest.skip("identical to the plain path")
    if mode == 0 and compact == 0:
        pytest.skip("no entry threshold: nothing to compact")
    rng = np.random.default_rng(shape[0] * 13 + shape[1] + 7 * tkind)
    X = smooth_matrix(rng, *shape)
    if tkind == 0:
        # two disjoint row/column blocks: the Gram matrix has exact zeros
        m, n = shape
        X[: m // 2, n // 2:] = 0.0
        X[m // 2:, : n // 2] = 0.0
    p = min(shape)
    T = transform(tkind, p)
    Phi = O.phi(X, T)
    if mode == 0:
        eps, arg = -1.0, 0.0
    else:
        eps, k, ratio = gap_threshold(Phi)
        assert ratio > 1.02   # FP32 Phi is accurate to ~1e-6: the same entries survive
        arg = eps if mode == 1 else (k - 0.5) / (p * p)   # ceil(frac p^2) = k
    Phib = np.where(np.abs(Phi) >= eps, Phi, 0.0) if eps >= 0 else Phi
    lam = 1.05 * np.max(np.abs(np.linalg.eigvalsh(Phib)))
    s = O.Shrink(O.SOFT, 0.1 * math.sqrt(lam))
    L = 15
    ref = O.cpa(X, s, L, lam, T=None if tkind == 0 else T, eps_thr=eps)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, compact)
    try:
        Y = cpa.cpa_svt(handle, Xd, {"kind": O.SOFT, "tau": s.tau}, L, lam, prec, sparsify=(tkind, mode, arg))
        torch.cuda.synchronize()
    finally:
        cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, 1)
    got = Y.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL[prec], (shape, tkind, mode, prec, compact, err)


def test_sparsify_argument_errors(cpa, handle):
    import torch
    X = torch.randn((20, 10), device="cuda")
    for bad in [(5, 0, 0.0), (0, 3, 0.0), (0, 1, -1.0), (0, 2, 0.0), (0, 2, 1.5)]:
        with pytest.raises(cpa.CpaError):
            cpa.cpa_svt(handle, X, {"kind": O.SOFT, "tau": 1.0}, 5, 10.0, "fp32", sparsify=bad)


_PHI_CACHE = {}


def _big_case(tkind):
    """The smooth 1100 x 1024 matrix (p = 1024: the multi-block top-k search
    and the large-size transforms run) and the oracle's Phi for transform
    tkind, computed once per transform."""
    if tkind not in _PHI_CACHE:
        rng = np.random.default_rng(4242 + tkind)
        X = smooth_matrix(rng, 1100, 1024)
        if tkind == 0:
            X[:550, 512:] = 0.0
            X[550:, :512] = 0.0
        T = transform(tkind, 1024)
        _PHI_CACHE[tkind] = (X, T, O.phi(X, T if tkind else None))
    return _PHI_CACHE[tkind]


def wide_gap(Phi, lo_frac=0.0005, hi_frac=0.5):
    """eps in the widest multiplicative gap of |Phi| within a rank window
    (vectorised form of gap_threshold for large p)."""
    a = np.sort(np.abs(Phi).ravel())[::-1]
    lo, hi = max(1, int(lo_frac * a.size)), int(hi_frac * a.size)
    seg = a[lo - 1:hi]
    pos = seg[1:] > 0
    if not np.all(pos):   # exact zeros (block-structured Phi): keep every nonzero
        k = lo + int(np.argmin(pos))
        return 0.5 * a[k - 1], k, math.inf
    r = seg[:-1] / seg[1:]
    j = int(np.argmax(r))
    k = lo + j
    return math.sqrt(a[k - 1] * a[k]), k, float(r[j])


@pytest.mark.parametrize("tkind", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("compact", [1, 0])
def test_sparsify_full_size_sampled(cpa, handle, tkind, mode, prec, compact):
    """p = 1024 with every transform and both threshold modes: sampled rows
    of X T^T H_hat(Phi_) T against the oracle (Phi from the C oracle, the
    series on the sampled rows by the oracle's block vector form)."""
    import torch
    X, T, Phi = _big_case(tkind)
    p = 1024
    eps, k, ratio = wide_gap(Phi)
    assert ratio > 1.02
    arg = eps if mode == 1 else (k - 0.5) / (p * p)
    Phib = np.where(np.abs(Phi) >= eps, Phi, 0.0)
    lam = 1.05 * np.max(np.abs(np.linalg.eigvalsh(Phib)))
    s = O.Shrink(O.SOFT, 0.1 * math.sqrt(lam))
    L = 15
    rows = [0, 1, 550, 1098, 1099]
    want = (T.T @ O.filter_block(Phib, s, L, lam, T @ X[rows].T)).T
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, compact)
    try:
        Y = cpa.cpa_svt(handle, Xd, {"kind": O.SOFT, "tau": s.tau}, L, lam, prec, sparsify=(tkind, mode, arg))
        torch.cuda.synchronize()
    finally:
        cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, 1)
    got = Y.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(got) / np.sqrt(len(got))
    for j, i in enumerate(rows):
        err = np.linalg.norm(got[i] - want[j]) / max(np.linalg.norm(want[j]), scale)
        assert err <= TOL[prec], (tkind, mode, prec, compact, i, err, k)


@pytest.mark.parametrize("tkind", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [1, 2])
def test_zero_tile_skip_is_bit_identical(cpa, handle, tkind, mode):
    """The recurrence on the full thresholded operand (no compaction) skips
    its all-zero tiles: the same result, bit for bit, as running every tile
    (the skipped products are exact zeros)."""
    import torch
    from paper_1705_07112_gb300 import _lib
    X, T, Phi = _big_case(tkind)
    p = 1024
    eps, k, _ = wide_gap(Phi)
    arg = eps if mode == 1 else (k - 0.5) / (p * p)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    lam = 1.05 * np.max(np.abs(np.linalg.eigvalsh(np.where(np.abs(Phi) >= eps, Phi, 0.0))))
    spec = {"kind": O.SOFT, "tau": 0.1 * math.sqrt(lam)}
    out = []
    _lib.cpa_set_option(handle, _lib.OPT_SPARSE_COMPACT, 0)
    try:
        for skip in (1, 0):
            _lib.cpa_set_option(handle, _lib.OPT_SPARSE_SKIP, skip)
            Y = cpa.cpa_svt(handle, Xd, spec, 15, lam, "bf16x3", sparsify=(tkind, mode, arg))
            torch.cuda.synchronize()
            out.append(Y.cpu().numpy())
    finally:
        _lib.cpa_set_option(handle, _lib.OPT_SPARSE_SKIP, 1)
        _lib.cpa_set_option(handle, _lib.OPT_SPARSE_COMPACT, 1)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("shape", [(120, 64), (64, 120), (90, 37)])
@pytest.mark.parametrize("tkind", [2, 3])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("compact", [1, 0])
def test_guarded_interval_matches_oracle(cpa, handle, shape, tkind, mode, prec, compact):
    """The guarded interval [-|Phi - Phi_|_F, Lambda_max] for the
    thresholded Phi_ (cpa_sparsify.interval = 1) against the oracle's
    guarded form (oracle/interval.py) with the same T, eps and Lambda_max."""
    import torch
    from oracle import interval as I
    rng = np.random.default_rng(shape[0] * 7 + shape[1] + 3 * tkind)
    X = smooth_matrix(rng, *shape)
    p = min(shape)
    T = transform(tkind, p)
    Phi = O.phi(X, T)
    eps, k, ratio = gap_threshold(Phi)
    assert ratio > 1.02
    arg = eps if mode == 1 else (k - 0.5) / (p * p)
    lam = 1.05 * np.max(np.abs(np.linalg.eigvalsh(np.where(np.abs(Phi) >= eps, Phi, 0.0))))
    s = O.Shrink(O.SOFT, 0.1 * math.sqrt(lam))
    L = 15
    ref = I.guarded_cpa(X, s, L, lam, T, eps)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, compact)
    try:
        Y = cpa.cpa_svt(handle, Xd, {"kind": O.SOFT, "tau": s.tau}, L, lam, prec, sparsify=(tkind, mode, arg, 1))
        torch.cuda.synchronize()
    finally:
        cpa._lib.cpa_set_option(handle, cpa._lib.OPT_SPARSE_COMPACT, 1)
    got = Y.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL[prec], (shape, tkind, mode, prec, compact, err)
    # the unguarded result differs where Phi_ has negative eigenvalues
    if np.min(np.linalg.eigvalsh(np.where(np.abs(Phi) >= eps, Phi, 0.0))) < -1e-6 * lam:
        plain = O.cpa(X, s, L, lam, T=T, eps_thr=eps)
        assert np.linalg.norm(plain - ref) > 0.0
    with pytest.raises(cpa.CpaError):
        cpa.cpa_svt(handle, Xd, {"kind": O.SOFT, "tau": s.tau}, L, lam, prec, sparsify=(tkind, mode, arg, 2))
