"""The predictor's training labels and its FP64 feature restatement
(tests/predictor_data.py), pinned on the CPU against the dense oracle and
against spectral facts."""
import math

import numpy as np

import oracle as O
import predictor_data as D


def test_spectral_errors_match_the_oracle_series():
    """The vectorised Chebyshev evaluation of the labels equals the oracle's
    own series recurrence route (approx_error_spectral)."""
    mats, specs = D.generate(6, seed=31)
    for X, s in zip(mats, specs):
        Xd = X.astype(np.float64)
        m, n = X.shape
        _, _, sv = O.svd_jacobi(Xd if m >= n else Xd.T)
        lam = 1.02 * float(np.max(sv)) ** 2
        hx = np.array([O.h(s, v * v) for v in sv])
        denom = float(np.sqrt(np.sum((sv * hx) ** 2)))
        got = D.spectral_errors(sv, s, lam, [5, 17, 40])
        ref = [O.approx_error_spectral(sv, s, L, lam) / denom for L in (5, 17, 40)]
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-13)


def test_label_order_meets_the_tolerance_on_the_dense_oracle():
    """Brute force: Algorithm 1 in FP64 with the labelled L* (and the bound
    the label uses) is within TOL of the exact shrinkage, and L* - 1 is not
    (L* starts the run of passing orders that ends at 96)."""
    mats, specs = D.generate(40, seed=32)
    checked = 0
    for X, s in zip(mats, specs):
        t0, t1, sv = D.label(X, s)
        L = int(round(math.exp(t1)))
        if L > D.L_HI:
            continue
        Xd = X.astype(np.float64)
        p = min(X.shape)
        lam = O.lambda_bound(Xd, D.POWER_ITERS, D.MARGIN, O.start_vector(D.START_SEED, p))["lam"]
        ex = O.shrink_exact(Xd, s)
        den = np.linalg.norm(ex)
        assert np.linalg.norm(O.cpa(Xd, s, L, lam) - ex) / den <= D.TOL
        if L > D.L_LO:
            assert np.linalg.norm(O.cpa(Xd, s, L - 1, lam) - ex) / den > D.TOL
        assert t0 >= -1e-12   # theta_4 <= sigma_max^2
        checked += 1
        if checked == 6:
            break
    assert checked >= 3


def test_reference_features_obey_spectral_bounds():
    mats, specs = D.generate(20, seed=33)
    for X, s in zip(mats, specs):
        f = D.reference_features(X, s)
        Xd = X.astype(np.float64)
        m, n = X.shape
        sv = np.linalg.svd(Xd, compute_uv=False)
        E = float(np.sum(sv ** 2))
        th4 = E / math.exp(f[2])
        lmin = th4 * math.exp(f[4])
        assert th4 <= sv[0] ** 2 * (1 + 1e-12)
        assert lmin >= sv[-1] ** 2 * (1 - 1e-9) and lmin <= th4 * (1 + 1e-12)
        assert abs(math.exp(f[6]) * th4 ** 2 - np.sum(sv ** 4)) <= 1e-9 * np.sum(sv ** 4)
        assert f[0] == math.log(min(m, n)) and f[1] == math.log(max(m, n) / min(m, n))
        assert f[8] >= -1e-12   # Rayleigh quotients grow along the power iteration
        assert (f[10], f[11]) == ((1.0, 0.0) if s.kind == O.HARD else (0.0, 1.0) if s.kind == O.WSOFT
                                  else (0.0, 0.0))
