"""Pins of the guarded series interval (oracle/interval.py): with a = 0 it
is the C oracle's Algorithm 1 (an independent implementation), its
coefficients interpolate h at the nodes mapped to [a, b], the filter it
builds equals the spectral definition through LAPACK's eigendecomposition
of the thresholded Phi, Weyl's bound holds for the lower end, and on a
spectrum that reaches below zero the guarded filter stays bounded where
the unguarded one does not."""
import math

import numpy as np

import oracle as O
from oracle import interval as I

RNG = np.random.default_rng(1705)


def rand_orth(p):
    Q, R = np.linalg.qr(RNG.standard_normal((p, p)))
    return Q * np.sign(np.diag(R))


def test_zero_lower_end_is_algorithm_1():
    X = RNG.standard_normal((23, 17))
    T = rand_orth(17)
    lam = 1.05 * np.linalg.norm(X, 2) ** 2
    for kind in (O.HARD, O.SOFT, O.WSOFT):
        s = O.Shrink(kind, 2.0, c=4.0, eps=1e-8, noise=1.0)
        assert np.allclose(I.coeffs_interval(s, 12, 0.0, lam), O.coeffs(s, 12, lam), rtol=0, atol=1e-12)
        for L in (1, 2, 5, 20):
            for eps in (-1.0, 0.5):
                for A in (X, X.T):
                    got = I.cpa_interval(A, s, L, 0.0, lam, T, eps)
                    ref = O.cpa(A, s, L, lam, T=T, eps_thr=eps)
                    assert np.allclose(got, ref, rtol=0, atol=1e-10 * max(1.0, np.abs(ref).max()))


def test_coefficients_interpolate_h_on_the_interval():
    s = O.Shrink(O.SOFT, 1.3)
    for (a, b) in ((-4.0, 30.0), (0.0, 9.0), (-0.5, 2.0)):
        for L in (3, 8, 21):
            c = I.coeffs_interval(s, L, a, b)
            ck = c.copy()
            ck[0] *= 0.5
            for l in range(1, L + 1):
                y = math.cos(math.pi * (l - 0.5) / L)
                x = a + 0.5 * (b - a) * (y + 1.0)
                want = O.h(s, x) if x > 0 else 0.0
                assert abs(np.polynomial.chebyshev.chebval(y, ck) - want) < 1e-12


def test_filter_equals_the_spectral_definition():
    """H = Q diag(h_hat(mu)) Q^T for Phi_ = Q diag(mu) Q^T (LAPACK eigh),
    h_hat the scalar series on [a, b]."""
    X = RNG.standard_normal((30, 12)) @ np.diag(np.linspace(0.2, 3.0, 12))
    T = rand_orth(12)
    G = X.T @ X
    Phi = T @ G @ T.T
    eps = np.quantile(np.abs(Phi), 0.6)
    Phs = I.threshold(Phi, eps)
    a = -I.removed_norm(Phi, eps)
    b = 1.05 * np.linalg.eigvalsh(Phs).max()
    s = O.Shrink(O.SOFT, 1.0)
    L = 25
    _, H = I.cpa_interval(X, s, L, a, b, T, eps, return_H=True)
    mu, Q = np.linalg.eigh(Phs)
    ck = I.coeffs_interval(s, L, a, b)
    ck[0] *= 0.5
    hh = np.polynomial.chebyshev.chebval((2.0 * mu - (a + b)) / (b - a), ck)
    assert np.allclose(H, Q @ np.diag(hh) @ Q.T, atol=1e-10 * max(1.0, np.abs(hh).max()))


def test_weyl_bound_for_the_lower_end():
    for trial in range(20):
        p = int(RNG.integers(4, 40))
        X = RNG.standard_normal((p + 5, p))
        Phi = X.T @ X
        eps = np.quantile(np.abs(Phi), RNG.uniform(0.2, 0.95))
        mu_min = np.linalg.eigvalsh(I.threshold(Phi, eps)).min()
        assert mu_min >= -I.removed_norm(Phi, eps) - 1e-9 * np.abs(Phi).max()


def test_guard_keeps_the_series_bounded_below_zero():
    """A thresholded Phi_ with a clearly negative eigenvalue: on [0, b] the
    series is evaluated outside its interval there and grows with L; on
    [a, b] it stays within the response's range."""
    # Phi = u u^T, u = (1, 0.3, ..., 0.3): the threshold 0.1 keeps the
    # first row and column and drops every 0.09 entry, diagonal included,
    # leaving an arrow matrix with eigenvalues (1 +- sqrt(1 + 4 * 0.09 * 15)) / 2
    p = 16
    u = np.full(p, 0.3)
    u[0] = 1.0
    Phi = np.outer(u, u)
    eps = 0.1
    Phs = I.threshold(Phi, eps)
    mu = np.linalg.eigvalsh(Phs)
    assert mu.min() < -0.05 * mu.max()
    a = -I.removed_norm(Phi, eps)
    b = 1.05 * mu.max()
    s = O.Shrink(O.SOFT, 0.5)
    L = 40
    Hg = I.filter_matrix(Phs, I.coeffs_interval(s, L, a, b), a, b)
    Hu = I.filter_matrix(Phs, I.coeffs_interval(s, L, 0.0, b), 0.0, b)
    # h lies in [0, 1): the guarded filter's spectrum stays near that range
    assert np.abs(np.linalg.eigvalsh(Hg)).max() < 1.5
    assert np.abs(np.linalg.eigvalsh(Hu)).max() > 10.0


def test_interval_ends_and_convergence_to_h():
    """a Id and b Id go to T_k(-1) = (-1)^k and T_k(1) = 1; and for many
    terms the filter approaches h itself on the spectrum of a thresholded
    Phi (0 at its negative eigenvalues), which a wrong map of [a, b] onto
    [-1, 1] would not."""
    s = O.Shrink(O.SOFT, 0.4)
    a, b = -0.8, 2.0
    c = I.coeffs_interval(s, 15, a, b)
    ends = c.copy()
    ends[0] *= 0.5
    Ha = I.filter_matrix(a * np.eye(3), c, a, b)
    Hb = I.filter_matrix(b * np.eye(3), c, a, b)
    assert np.allclose(Ha, np.sum(ends * (-1.0) ** np.arange(15)) * np.eye(3), atol=1e-12)
    assert np.allclose(Hb, np.sum(ends) * np.eye(3), atol=1e-12)
    p = 16
    u = np.full(p, 0.3)
    u[0] = 1.0
    Phi = np.outer(u, u)
    Phs = I.threshold(Phi, 0.1)
    a = -I.removed_norm(Phi, 0.1)
    mu, Q = np.linalg.eigh(Phs)
    b = 1.05 * mu.max()
    H = I.filter_matrix(Phs, I.coeffs_interval(s, 400, a, b), a, b)
    hmu = np.array([O.h(s, x) if x > 0 else 0.0 for x in mu])
    assert np.abs(np.diag(Q.T @ H @ Q) - hmu).max() < 2e-2


def test_block_compaction_identity():
    """The identity the device's compaction of a thresholded operand rests
    on: for a symmetric Phi_ whose nonzero rows (and columns) are S, the
    series H_hat(Phi_) on [a, b] is H_hat(Phi_[S, S]) on S x S, zero between
    S and its complement, and c_out Id on the complement with c_out the
    series at the scalar -sigma, sigma = (a + b) / (b - a); the transformed
    filter T^T H T is T_S^T (H_hat(Phi_[S,S]) - c_out Id) T_S + c_out T^T T.
    Checked on both the plain interval [0, b] and a guarded one, for an
    orthonormal T (DCT by QR of a random matrix) and the masked Haar T."""
    p = 23
    S = np.array([1, 4, 5, 11, 17, 22])
    B = RNG.standard_normal((len(S), len(S)))
    A = B @ B.T - 0.3 * np.eye(len(S))   # a spectrum reaching below zero, inside [a, b] below
    Phi = np.zeros((p, p))
    Phi[np.ix_(S, S)] = A
    rest = np.setdiff1d(np.arange(p), S)
    Q = rand_orth(p)
    haar = np.zeros((p, p))
    for i in range(p // 2):
        haar[i, 2 * i] = haar[i, 2 * i + 1] = math.sqrt(0.5)
    haar[p // 2, p - 1] = 1.0
    s = O.Shrink(O.SOFT, 0.7)
    lam = 1.02 * np.max(np.linalg.eigvalsh(A))
    for (a, b) in ((0.0, lam), (-0.8, lam)):
        for L in (1, 2, 3, 9, 16):
            c = I.coeffs_interval(s, L, a, b)
            Hf = I.filter_matrix(Phi, c, a, b)
            Hb = I.filter_matrix(A, c, a, b)
            ck = c.copy()
            ck[0] *= 0.5
            c_out = np.polynomial.chebyshev.chebval(-(a + b) / (b - a), ck)
            assert np.allclose(Hf[np.ix_(S, S)], Hb, rtol=0, atol=1e-12)
            assert np.allclose(Hf[np.ix_(S, rest)], 0.0, rtol=0, atol=1e-12)
            assert np.allclose(Hf[np.ix_(rest, rest)], c_out * np.eye(len(rest)), rtol=0, atol=1e-12)
            for T in (Q, haar):
                TS = T[S]
                want = T.T @ Hf @ T
                got = TS.T @ (Hb - c_out * np.eye(len(S))) @ TS + c_out * (T.T @ T)
                assert np.allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))
    # the masked Haar transform's T^T T: 1/2 on the 2 x 2 blocks of the
    # pairs (2i, 2i + 1) and 1 at (p - 1, p - 1) for odd p
    want = np.zeros((p, p))
    for i in range(p // 2):
        want[2 * i:2 * i + 2, 2 * i:2 * i + 2] = 0.5
    want[p - 1, p - 1] = 1.0
    assert np.allclose(haar.T @ haar, want, rtol=0, atol=1e-15)
