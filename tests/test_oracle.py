"""Pins of the FP64 oracle against mathematics it does not itself define.

Each test ties one oracle function to a closed form, an invariant, or an
independent library routine (numpy/scipy), chosen so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails at least one
of them.  Sizes are small: the whole file runs in seconds on a CPU.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import oracle as O

RNG = np.random.default_rng(20240601)


def rand_orth(rng, n):
    """Product of Householder reflectors of random unit vectors: a random
    orthogonal matrix built without any factorisation routine."""
    Q = np.eye(n)
    for _ in range(n):
        v = rng.standard_normal(n)
        v /= np.linalg.norm(v)
        Q = Q - 2.0 * np.outer(Q @ v, v)
    return Q


def hhat_closed(s: O.Shrink, alpha, lam, x):
    """h_hat(x) on [0, lam] evaluated with numpy's Chebyshev series routine
    on the oracle's coefficients (numpy's chebval uses the full c_0, the
    paper's series halves it)."""
    ck = O.coeffs(s, alpha, lam).copy()
    ck[0] *= 0.5
    return npcheb.chebval(2.0 * np.asarray(x) / lam - 1.0, ck)


# ---------------------------------------------------------------- scalar CPA

@pytest.mark.parametrize("k", [0, 1, 2, 3, 7, 20, 49])
def test_chebyshev_polynomial_is_cos_k_theta(k):
    # Eq. chebychev_polynomial vs the recurrence Eq. chebyche2: T_k(cos t) = cos(k t)
    for t in np.linspace(0.0, math.pi, 17):
        assert abs(O.cheb_T(k, math.cos(t)) - math.cos(k * t)) < 1e-12


@pytest.mark.parametrize("alpha", [1, 2, 3, 8, 20])
def test_discrete_coefficients_recover_polynomials(alpha):
    # Eq. chebychev_coeff_discrete is exact for a degree <= alpha-1 polynomial.
    a = RNG.standard_normal(alpha)
    th = math.pi * (np.arange(1, alpha + 1) - 0.5) / alpha
    hs = npcheb.chebval(np.cos(th), a)           # library evaluation
    ck = O.coeffs_from_nodes(hs)
    want = a.copy()
    want[0] *= 2.0                                # series uses c_0 / 2
    assert np.allclose(ck, want, atol=1e-12)


def test_discrete_coefficients_of_exp_match_bessel():
    # Closed form: e^x = I_0(1) + 2 sum_k I_k(1) T_k(x), so c_k -> 2 I_k(1).
    special = pytest.importorskip("scipy.special")
    alpha = 20
    th = math.pi * (np.arange(1, alpha + 1) - 0.5) / alpha
    ck = O.coeffs_from_nodes(np.exp(np.cos(th)))
    want = 2.0 * special.iv(np.arange(alpha), 1.0)
    assert np.allclose(ck, want, atol=1e-14)


@pytest.mark.parametrize("alpha", [2, 5, 20, 31])
def test_series_forms_agree_with_library(alpha):
    ck = RNG.standard_normal(alpha)
    lib = ck.copy()
    lib[0] *= 0.5
    for x in np.linspace(-1, 1, 13):
        a = O.series_cos(ck, x)
        b = O.series_rec(ck, x)
        c = npcheb.chebval(x, lib)
        assert abs(a - c) < 1e-11 and abs(b - c) < 1e-11


def shrinks():
    return [O.Shrink(O.HARD, 1.3), O.Shrink(O.SOFT, 0.7),
            O.Shrink(O.WSOFT, 0.0, c=0.3, eps=1e-8, noise=0.2)]


def test_responses_special_cases():
    # Eq. filter_response_ours: hard -> 0/1 step, soft -> max(sigma - tau, 0)
    hard, soft, ws = shrinks()
    for sig in [0.0, 0.5, 1.29, 1.3, 1.31, 2.0, 10.0]:
        assert O.g(hard, sig) == (sig if sig > 1.3 else 0.0)
        assert abs(O.g(soft, sig) - max(sig - 0.7, 0.0)) < 1e-15
    # weighted soft: g(sigma) = max(sigma - w, 0), w = c/(sqrt(sigma^2 - noise) + eps)
    for sig in [0.3, 0.5, 0.7, 1.0, 3.0]:
        w = 0.3 / (math.sqrt(max(sig * sig - 0.2, 0.0)) + 1e-8)
        assert abs(O.g(ws, sig) - max(sig - w, 0.0)) < 1e-12
    # tie at the threshold is "otherwise" (strict >)
    assert O.h(O.Shrink(O.SOFT, 2.0), 4.0) == 0.0


@pytest.mark.parametrize("alpha", [3, 10, 24])
@pytest.mark.parametrize("lam", [1.0, 37.5])
def test_shifted_coefficients_interpolate_at_nodes(alpha, lam):
    # The alpha-term series with the discrete coefficients interpolates h at
    # the alpha shifted Chebyshev nodes (discrete orthogonality of cos k theta).
    for s in shrinks():
        ck = O.coeffs(s, alpha, lam)
        for l in range(1, alpha + 1):
            th = math.pi * (l - 0.5) / alpha
            x = 0.5 * lam * (math.cos(th) + 1.0)
            assert abs(O.series_rec(ck, math.cos(th)) - O.h(s, x)) < 1e-11


def test_soft_series_converges_with_order():
    s = O.Shrink(O.SOFT, 0.5)
    lam = 4.0
    xs = np.linspace(0.0, lam, 401)
    exact = np.array([O.h(s, x) for x in xs])
    errs = []
    for alpha in [10, 20, 40, 80]:
        errs.append(np.max(np.abs(hhat_closed(s, alpha, lam, xs[xs > 1.0]) - exact[xs > 1.0])))
    assert errs[0] > errs[1] > errs[2] > errs[3]


# ---------------------------------------------------------------- SVD / EVD

def test_jacobi_svd_closed_forms():
    # diagonal
    d = np.array([3.0, -2.0, 0.5, 0.0])
    X = np.zeros((6, 4))
    X[:4, :4] = np.diag(d)
    W, V, s = O.svd_jacobi(X)
    assert np.allclose(np.sort(s), np.sort(np.abs(d)), atol=1e-14)
    # rank one: 5 u v^T
    u = RNG.standard_normal(7); u /= np.linalg.norm(u)
    v = RNG.standard_normal(5); v /= np.linalg.norm(v)
    W, V, s = O.svd_jacobi(5.0 * np.outer(u, v))
    assert np.allclose(np.sort(s), [0, 0, 0, 0, 5.0], atol=1e-12)
    # Q1 diag(s) Q2^T with known s
    Q1, Q2 = rand_orth(RNG, 9), rand_orth(RNG, 6)
    sv = np.array([10.0, 4.0, 2.5, 1.0, 0.1, 0.01])
    X = Q1[:, :6] @ np.diag(sv) @ Q2.T
    W, V, s = O.svd_jacobi(X)
    assert np.allclose(np.sort(s)[::-1], sv, rtol=1e-12)
    assert np.allclose(V.T @ V, np.eye(6), atol=1e-13)
    assert np.allclose(W @ V.T, X, atol=1e-12)


def test_jacobi_svd_matches_lapack():
    X = RNG.standard_normal((40, 25))
    _, _, s = O.svd_jacobi(X)
    assert np.allclose(np.sort(s)[::-1], np.linalg.svd(X, compute_uv=False), rtol=1e-11)


def test_jacobi_eig_matches_lapack():
    A = RNG.standard_normal((30, 30))
    S = A + A.T
    w, V = O.eig_jacobi(S)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(S), atol=1e-11)
    assert np.allclose(V @ np.diag(w) @ V.T, S, atol=1e-11)


@pytest.mark.parametrize("shape", [(30, 20), (20, 30), (16, 16)])
def test_exact_shrink_three_ways(shape):
    # SVD-based (Eq. sing_shrink_exact), EVD-based (Eq. sing_shrink_exact_from_eig2)
    # and LAPACK's SVD with the scalar g applied agree.
    X = RNG.standard_normal(shape)
    for s in shrinks():
        a = O.shrink_exact(X, s)
        b = O.shrink_exact_evd(X, s)
        U, sv, Vt = np.linalg.svd(X, full_matrices=False)
        c = U @ np.diag([O.g(s, x) for x in sv]) @ Vt
        assert np.allclose(a, c, atol=1e-10), s
        assert np.allclose(b, c, atol=1e-8), s


# ---------------------------------------------------------------- matrix CPA

@pytest.mark.parametrize("kind", [O.HARD, O.SOFT, O.WSOFT])
@pytest.mark.parametrize("shape", [(12, 8), (8, 12), (10, 10)])
def test_cpa_closed_form_known_svd(kind, shape):
    # X = Q1 diag(s) Q2^T  =>  CPA(X) = Q1 diag(s_i h_hat(s_i^2)) Q2^T  (Eq. ATA_eig_fil, T = Id)
    m, n = shape
    p = min(m, n)
    Q1, Q2 = rand_orth(RNG, m), rand_orth(RNG, n)
    sv = np.linspace(3.0, 0.2, p)
    X = Q1[:, :p] @ np.diag(sv) @ Q2[:, :p].T
    s = {O.HARD: O.Shrink(O.HARD, 1.1), O.SOFT: O.Shrink(O.SOFT, 0.9),
         O.WSOFT: O.Shrink(O.WSOFT, 0.0, c=0.5, eps=1e-8, noise=0.1)}[kind]
    lam, alpha = 10.0, 17
    Y = O.cpa(X, s, alpha, lam)
    want = Q1[:, :p] @ np.diag(sv * hhat_closed(s, alpha, lam, sv ** 2)) @ Q2[:, :p].T
    assert np.allclose(Y, want, atol=1e-11)


def test_cpa_diagonal_input():
    d = np.array([4.0, 3.0, 1.0, 0.5, 0.0])
    X = np.diag(d)
    s = O.Shrink(O.SOFT, 0.8)
    Y = O.cpa(X, s, 12, 20.0)
    assert np.allclose(Y, np.diag(d * hhat_closed(s, 12, 20.0, d ** 2)), atol=1e-12)


@pytest.mark.parametrize("alpha", [1, 2, 3, 9])
def test_cpa_brute_force_tiny(alpha):
    # Brute force through LAPACK's eigendecomposition of X^T X (p <= 6).
    X = RNG.standard_normal((9, 6))
    s = O.Shrink(O.SOFT, 1.0)
    lam = 1.05 * np.linalg.norm(X, 2) ** 2
    w, V = np.linalg.eigh(X.T @ X)
    want = X @ V @ np.diag(hhat_closed(s, alpha, lam, w)) @ V.T
    assert np.allclose(O.cpa(X, s, alpha, lam), want, atol=1e-11)


def test_cpa_invariances():
    X = RNG.standard_normal((14, 9))
    s = O.Shrink(O.SOFT, 1.2)
    lam = 1.1 * np.linalg.norm(X, 2) ** 2
    Y = O.cpa(X, s, 15, lam)
    # transpose: CPA(X^T) = CPA(X)^T
    assert np.allclose(O.cpa(X.T, s, 15, lam), Y.T, atol=1e-11)
    # orthogonal invariance: CPA(Q1 X Q2) = Q1 CPA(X) Q2
    Q1, Q2 = rand_orth(RNG, 14), rand_orth(RNG, 9)
    assert np.allclose(O.cpa(Q1 @ X @ Q2, s, 15, lam), Q1 @ Y @ Q2, atol=1e-10)
    # zero padding contributes nothing (rows of zeros, columns of zeros)
    Xp = np.zeros((20, 9)); Xp[:14] = X
    assert np.allclose(O.cpa(Xp, s, 15, lam)[:14], Y, atol=1e-11)
    assert np.allclose(O.cpa(Xp, s, 15, lam)[14:], 0.0, atol=0)
    # scaling: CPA(a X; a^2 lam, a tau) = a CPA(X; lam, tau) for hard and soft
    for kind in [O.HARD, O.SOFT]:
        s1 = O.Shrink(kind, 1.2)
        s2 = O.Shrink(kind, 1.2 * 3.0)
        assert np.allclose(O.cpa(3.0 * X, s2, 15, 9.0 * lam), 3.0 * O.cpa(X, s1, 15, lam), atol=1e-10)


def test_cpa_error_identity_against_exact():
    # |CPA(X) - G(X)|_F computed from the spectrum equals the matrix difference.
    X = RNG.standard_normal((30, 18))
    for s in shrinks():
        lam = 1.02 * np.linalg.norm(X, 2) ** 2
        Y = O.cpa(X, s, 20, lam)
        E = O.shrink_exact(X, s)
        sv = np.linalg.svd(X, compute_uv=False)
        assert abs(np.linalg.norm(Y - E) - O.approx_error_spectral(sv, s, 20, lam)) < 1e-9


def test_cpa_approaches_exact_for_soft():
    X = RNG.standard_normal((24, 16))
    s = O.Shrink(O.SOFT, 2.0)
    lam = 1.02 * np.linalg.norm(X, 2) ** 2
    E = O.shrink_exact(X, s)
    errs = [np.linalg.norm(O.cpa(X, s, a, lam) - E) for a in (5, 20, 80)]
    assert errs[0] > errs[1] > errs[2]


def test_cpa_vec_matches_dense_rows_and_columns():
    s = O.Shrink(O.SOFT, 1.0)
    for shape in [(15, 9), (9, 15)]:
        X = RNG.standard_normal(shape)
        lam = 1.1 * np.linalg.norm(X, 2) ** 2
        Y, H = O.cpa(X, s, 11, lam, return_H=True)
        m, n = shape
        if m >= n:   # Y = X H: row i of Y = H x_i
            for i in [0, 4, m - 1]:
                assert np.allclose(O.cpa_vec(X, s, 11, lam, X[i]), Y[i], atol=1e-11)
        else:        # Y = H X: column j of Y = H x_j
            for j in [0, 3, n - 1]:
                assert np.allclose(O.cpa_vec(X, s, 11, lam, X[:, j]), Y[:, j], atol=1e-11)
        # H itself: H e_j
        e = np.zeros(min(m, n)); e[2] = 1.0
        assert np.allclose(O.cpa_vec(X, s, 11, lam, e), H[:, 2], atol=1e-11)


def test_cpa_sparsity_options_reduce_to_dense():
    X = RNG.standard_normal((16, 12))
    s = O.Shrink(O.SOFT, 1.0)
    lam = 1.1 * np.linalg.norm(X, 2) ** 2
    Y = O.cpa(X, s, 13, lam)
    # eps = 0 keeps every entry (Eq. threshold_components)
    assert np.allclose(O.cpa(X, s, 13, lam, eps_thr=0.0), Y, atol=1e-12)
    # T = Id
    assert np.allclose(O.cpa(X, s, 13, lam, T=np.eye(12)), Y, atol=1e-12)
    # any orthogonal T without thresholding gives the same result (Eq. sing_shrink_exact_sparse)
    T = rand_orth(RNG, 12)
    assert np.allclose(O.cpa(X, s, 13, lam, T=T), Y, atol=1e-10)
    # a huge eps removes every entry: Phi_ = 0, B_hat = -Id, H = h_hat(0) Id
    Yz = O.cpa(X, s, 13, lam, eps_thr=1e30)
    assert np.allclose(Yz, X * hhat_closed(s, 13, lam, 0.0), atol=1e-12)


def test_lambda_bound_properties():
    X = RNG.standard_normal((50, 30))
    smax2 = np.linalg.norm(X, 2) ** 2
    v0 = O.start_vector(7, 30)
    r = O.lambda_bound(X, 20, 0.01, v0)
    assert r["theta"] <= smax2 * (1 + 1e-12)
    assert r["lam"] >= smax2
    assert abs(r["trace"] - np.sum(X * X)) < 1e-9
    assert r["lam"] <= r["trace"]
    # a rank-one X converges in one step to theta = sigma^2, residual 0
    u = RNG.standard_normal(20); v = RNG.standard_normal(10)
    X1 = np.outer(u, v)
    r1 = O.lambda_bound(X1, 3, 0.0, O.start_vector(1, 10))
    s2 = (np.linalg.norm(u) * np.linalg.norm(v)) ** 2
    assert abs(r1["theta"] - s2) < 1e-9 * s2 and r1["resid"] < 1e-6 * s2


def test_lambda_bound_exact_two_eigenvalue_closed_form():
    """The bound's value, not only its inequalities.  X = Q1 diag(s) Q2^T
    with two nonzero singular values and a start vector a q1 + b q2 in the
    span of their right singular vectors q1, q2: after t normalised
    products v = (alpha, beta) in that basis with alpha : beta =
    a mu1^t : b mu2^t (mu = s^2), so theta = alpha^2 mu1 + beta^2 mu2 and
    G v - theta v = (mu1 - mu2) alpha beta (beta, -alpha), whose norm is
    r = |mu1 - mu2| |alpha beta|.  The bound is min((theta + r) (1 +
    margin), mu1 + mu2).  A dropped residual, a dropped or doubled margin,
    an off-by-one iteration count or a wrong clamp each miss by far more
    than the 1e-12 asserted."""
    rng = np.random.default_rng(31)
    m, n = 9, 6
    Q1, Q2 = rand_orth(rng, m), rand_orth(rng, n)
    for (s1, s2, a, b, t, margin) in [(3.0, 2.0, 0.3, 0.9, 0, 0.01), (3.0, 2.0, 0.3, 0.9, 1, 0.01),
                                      (3.0, 2.0, 0.3, 0.9, 4, 0.01), (5.0, 4.5, -0.7, 0.2, 2, 0.01),
                                      (2.0, 1.0, 1.0, 1.0, 3, 0.05), (1.5, 1.4, 0.01, 1.0, 1, 0.0)]:
        S = np.zeros((m, n))
        S[0, 0], S[1, 1] = s1, s2
        X = Q1 @ S @ Q2.T
        v0 = a * Q2[:, 0] + b * Q2[:, 1]
        mu1, mu2 = s1 * s1, s2 * s2
        al, be = a * mu1 ** t, b * mu2 ** t
        nrm = np.hypot(al, be)
        al, be = al / nrm, be / nrm
        theta = al * al * mu1 + be * be * mu2
        r = abs(mu1 - mu2) * abs(al * be)
        want = min((theta + r) * (1.0 + margin), mu1 + mu2)
        got = O.lambda_bound(X, t, margin, v0)
        assert abs(got["theta"] - theta) <= 1e-12 * mu1, (t, got, theta)
        assert abs(got["resid"] - r) <= 1e-12 * mu1, (t, got, r)
        assert abs(got["trace"] - (mu1 + mu2)) <= 1e-12 * mu1
        assert abs(got["lam"] - want) <= 1e-12 * mu1, (t, got["lam"], want)
    # the trace clamp: a rank-one X gives theta = mu, r = 0, and (1 + margin)
    # mu exceeds the trace mu, so the bound is the trace itself
    X1 = np.outer(Q1[:, 0], Q2[:, 0]) * 2.5
    got = O.lambda_bound(X1, 2, 0.01, Q2[:, 0] + 0.5 * Q2[:, 3])
    assert abs(got["lam"] - 6.25) <= 1e-12 * 6.25 and abs(got["theta"] - 6.25) <= 1e-12 * 6.25


def test_start_vector_is_splitmix64():
    # SplitMix64 reference outputs for seed 0 (the published generator's
    # first outputs), top 53 bits scaled to [0,1) minus 1/2.
    first = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    want = [(z >> 11) / 2.0 ** 53 - 0.5 for z in first]
    assert np.allclose(O.start_vector(0, 3), want, atol=0)


def test_phi_is_the_transformed_gram():
    X = RNG.standard_normal((11, 7))
    T = rand_orth(RNG, 7)
    assert np.allclose(O.phi(X), X.T @ X, atol=1e-12)
    assert np.allclose(O.phi(X, T), T @ X.T @ X @ T.T, atol=1e-12)
    assert np.allclose(O.phi(X.T, T), T @ X.T @ X @ T.T, atol=1e-12)


def test_mlp_oracle_gradients_match_finite_differences():
    from oracle import mlp as M
    sizes = (5, 7, 6, 2)
    n = 7 * 5 + 7 + 6 * 7 + 6 + 2 * 6 + 2
    rng = np.random.default_rng(5)
    params = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((9, 5))
    T = rng.standard_normal((9, 2))
    g = M.gradients(params, sizes, X, T)
    h = 1e-6
    for i in range(n):
        e = np.zeros(n); e[i] = h
        fd = (M.loss(params + e, sizes, X, T) - M.loss(params - e, sizes, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # forward against an independent composition with explicit loops for one sample
    W1, b1, W2, b2, W3, b3 = M.unpack(params, sizes)
    x = X[3]
    a1 = [max(0.0, sum(W1[r, c] * x[c] for c in range(5)) + b1[r]) for r in range(7)]
    a2 = [max(0.0, sum(W2[r, c] * a1[c] for c in range(7)) + b2[r]) for r in range(6)]
    y = [sum(W3[r, c] * a2[c] for c in range(6)) + b3[r] for r in range(2)]
    assert np.allclose(M.forward(params, sizes, X)[0][3], y, atol=1e-12)


def test_adam_oracle_closed_forms():
    """With bias correction the first step moves each parameter by
    lr g/(|g|+eps), and so does every step of a constant gradient (the
    corrected moments then equal g and g^2 exactly); weight decay adds
    lr wd P."""
    from oracle import mlp as M
    rng = np.random.default_rng(12)
    P0 = rng.standard_normal(20)
    g = rng.standard_normal(20) * np.logspace(-3, 1, 20)
    lr, wd = 1e-2, 0.1
    opt = M.Adam(20)
    P1 = opt.step(P0, g, lr, wd)
    assert np.allclose(P1, P0 - lr * (g / (np.abs(g) + 1e-8) + wd * P0), rtol=0, atol=1e-14)
    opt = M.Adam(20)
    P = P0.copy()
    for _ in range(7):
        prev = P
        P = opt.step(P, g, lr, 0.0)
        assert np.allclose(P - prev, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
    # zero gradient, no decay: nothing moves
    assert np.array_equal(M.Adam(20).step(P0, np.zeros(20), lr, 0.0), P0)


def test_jacobi_svd_converges_on_rank_deficient_matrices():
    """Rank-1 and rank-2 inputs (numerically zero singular values): the
    Jacobi SVD converges and its singular values match the closed form."""
    u, v = RNG.standard_normal(60), RNG.standard_normal(50)
    for X, ref in ((np.full((60, 50), 4.0 / 3.0), [4.0 / 3.0 * np.sqrt(3000.0)]),
                   (np.outer(u, v), [np.linalg.norm(u) * np.linalg.norm(v)])):
        W, V, s = O.svd_jacobi(X, tol=60 * 2.220446049250313e-16)
        s = np.sort(s)[::-1]
        assert abs(s[0] - ref[0]) <= 1e-12 * ref[0]
        assert np.all(s[1:] <= 1e-12 * ref[0])
        Y = O.shrink_exact(X, O.Shrink(O.SOFT, 1.0))
        assert np.allclose(Y, X * (1.0 - 1.0 / ref[0]), atol=1e-12 * ref[0])
    A2 = RNG.standard_normal((40, 2)) @ RNG.standard_normal((2, 30))
    _, _, s = O.svd_jacobi(A2, tol=40 * 2.220446049250313e-16)
    ref = np.linalg.svd(A2, compute_uv=False)
    assert np.allclose(np.sort(s)[::-1][:2], ref[:2], rtol=1e-12)


def test_clenshaw_sum_equals_the_forward_recurrence():
    """Clenshaw's recurrence and Algorithm 1's forward recurrence sum the
    same truncated series: equal in FP64 for every kind, order and
    orientation, with and without a transform; on a 1 x 1 input both are
    x h_hat(x^2), the scalar series by cosines."""
    X = RNG.standard_normal((23, 17))
    T = rand_orth(RNG, 17)
    for kind in (O.HARD, O.SOFT, O.WSOFT):
        s = O.Shrink(kind, 2.0, c=4.0, eps=1e-8, noise=1.0)
        lam = 1.05 * np.linalg.norm(X, 2) ** 2
        for L in (1, 2, 3, 4, 9, 30):
            for A in (X, X.T):
                Yf, Hf = O.cpa(A, s, L, lam, return_H=True)
                Yc, Hc = O.cpa_clenshaw(A, s, L, lam, return_H=True)
                assert np.allclose(Hc, Hf, rtol=0, atol=1e-11 * max(1.0, np.abs(Hf).max()))
                assert np.allclose(Yc, Yf, rtol=0, atol=1e-11 * max(1.0, np.abs(Yf).max()))
            Yt = O.cpa_clenshaw(X, s, L, lam, T=T)
            assert np.allclose(Yt, O.cpa(X, s, L, lam, T=T), atol=1e-10)
    s = O.Shrink(O.SOFT, 0.7)
    for x in (0.3, 1.1, 2.5):
        ck = O.coeffs(s, 12, 9.0)
        y = O.cpa_clenshaw(np.array([[x]]), s, 12, 9.0)[0, 0]
        assert abs(y - x * O.series_cos(ck, 2 * x * x / 9.0 - 1)) < 1e-13


def test_block_vector_form_matches_the_c_oracle():
    """cpa_block (numpy matmul as the product) against the C oracle's
    one-vector form and dense Algorithm 1, both orientations, all kinds;
    filter_block on an explicit thresholded Phi against the dense
    Algorithm 1 with the same transform and entry threshold."""
    rng = np.random.default_rng(19)
    for (m, n) in [(23, 11), (11, 23), (9, 9)]:
        X = rng.standard_normal((m, n))
        p = min(m, n)
        lam = 1.02 * np.linalg.norm(X, 2) ** 2
        for s in (O.Shrink(O.SOFT, 1.1), O.Shrink(O.HARD, 1.3), O.Shrink(O.WSOFT, 0.0, 2.0, 1e-8, 0.5)):
            for alpha in (1, 2, 3, 14):
                V = rng.standard_normal((p, 4))
                B = O.cpa_block(X, s, alpha, lam, V)
                for j in range(4):
                    want = O.cpa_vec(X, s, alpha, lam, V[:, j])
                    assert np.allclose(B[:, j], want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))
                Y = O.cpa(X, s, alpha, lam)
                # rows (m >= n) or columns (m < n) of X H or H X
                Yb = O.cpa_block(X, s, alpha, lam, X.T if m >= n else X)
                assert np.allclose(Yb.T if m >= n else Yb, Y, rtol=0, atol=1e-11 * np.abs(Y).max())
    X = rng.standard_normal((20, 12))
    T = rand_orth(rng, 12)
    Phi = O.phi(X, T)
    eps = np.sort(np.abs(Phi).ravel())[-40]
    Phib = np.where(np.abs(Phi) >= eps, Phi, 0.0)
    lam = 1.05 * np.max(np.abs(np.linalg.eigvalsh(Phib)))
    s = O.Shrink(O.SOFT, 0.3 * np.sqrt(lam))
    Y = O.cpa(X, s, 11, lam, T=T, eps_thr=eps)
    # X T^T H(Phi_) T, row i = (T^T H T x_i)^T
    Yb = (T.T @ O.filter_block(Phib, s, 11, lam, T @ X.T)).T
    assert np.allclose(Yb, Y, rtol=0, atol=1e-11 * np.abs(Y).max())


def test_lapack_routes_match_the_jacobi_oracle():
    """singular_values and shrink_exact_lapack (LAPACK as the decomposition
    step) against the oracle's own one-sided Jacobi SVD and its exact
    shrinkage, and spectral_errors against the error of the dense FP64
    Algorithm 1 measured directly."""
    rng = np.random.default_rng(23)
    for shape in [(30, 17), (17, 30), (12, 12)]:
        X = rng.standard_normal(shape)
        _, _, sj = O.svd_jacobi(X if shape[0] >= shape[1] else X.T)
        assert np.allclose(O.singular_values(X), np.sort(sj)[::-1], rtol=1e-12, atol=1e-13)
        for s in shrinks():
            assert np.allclose(O.shrink_exact_lapack(X, s), O.shrink_exact(X, s), atol=1e-11)
            lam = 1.03 * O.singular_values(X)[0] ** 2
            want = [np.linalg.norm(O.cpa(X, s, a, lam) - O.shrink_exact(X, s)) /
                    np.linalg.norm(O.shrink_exact(X, s)) for a in (1, 2, 5, 17)]
            got = O.spectral_errors(O.singular_values(X), s, lam, [1, 2, 5, 17])
            assert np.allclose(got, want, rtol=1e-8, atol=1e-13), (s, got, want)
