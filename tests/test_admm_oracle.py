"""Pins of the FP64 background-modelling ADMM (oracle/admm.py) against the
mathematics it follows (the appendix ADMM Applicable Forms, Background Modeling, Eq. admm_algorithm_mod)."""
import numpy as np

import oracle as O
from oracle import admm as A

RNG = np.random.default_rng(1705)


def test_ls_update_is_the_least_squares_solution():
    """(K^T K)^{-1} K^T (z - u) equals the least-squares solution of
    K [l; s] = z - u computed by LAPACK on the stacked system."""
    n = 7
    z = [RNG.standard_normal(n) for _ in range(3)]
    u = [RNG.standard_normal(n) for _ in range(3)]
    I, Z0 = np.eye(n), np.zeros((n, n))
    K = np.block([[I, Z0], [Z0, I], [I, I]])
    rhs = np.concatenate([z[i] - u[i] for i in range(3)])
    ref = np.linalg.lstsq(K, rhs, rcond=None)[0]
    l, s = A.ls_update(*z, *u)
    assert np.allclose(np.concatenate([l, s]), ref, atol=1e-12)


def test_soft_is_the_l1_prox():
    """prox of t|.|_1 minimises t|y| + (y - x)^2 / 2: brute force on a grid."""
    xs = np.linspace(-3, 3, 13)
    grid = np.linspace(-4, 4, 80001)
    for t in (0.0, 0.5, 1.7):
        for x in xs:
            y = grid[np.argmin(t * np.abs(grid) + 0.5 * (grid - x) ** 2)]
            assert abs(A.soft(np.array([x]), t)[0] - y) <= 1e-4


def test_first_iterate_from_the_all_ones_start():
    """l_0 = s_0 = u_0 = 1, z_0 = K l'_0 = (1, 1, 2): a = (0, 0, 1), so
    l_1 = s_1 = 1/3 and E_1 = |1/3 - 1| / (1/3) = 2."""
    D = RNG.standard_normal((5, 4))
    seen = []

    def svt(X):
        seen.append(X.copy())
        return X
    A.rpca_admm(D, 0.1, 1, svt)
    assert np.allclose(seen[0], 1.0 / 3.0 + 1.0)
    _, _, E = A.rpca_admm(D, 0.1, 1, lambda X: X)
    assert abs(E[0] - 2.0) < 1e-12


def test_admm_recovers_low_rank_plus_sparse():
    """Textbook behaviour: on an incoherent rank-2 + 5 % sparse matrix the
    exact-SVT ADMM drives the constraint residual to zero and separates the
    parts (Candes, Li, Ma and Wright's regime; rho = mn / (4 |D|_1),
    eta = 1 / sqrt(max(m, n)))."""
    m, n = 60, 50
    L0 = RNG.standard_normal((m, 2)) @ RNG.standard_normal((2, n))
    S0 = np.zeros((m, n))
    mask = RNG.random((m, n)) < 0.05
    S0[mask] = RNG.choice([-1.0, 1.0], mask.sum()) * RNG.uniform(5, 10, mask.sum())
    D = L0 + S0
    rho = m * n / (4.0 * np.abs(D).sum())
    eta = 1.0 / np.sqrt(max(m, n))
    Lh, Sh, E = A.rpca_admm(D, eta / rho, 400, A.svt_exact(1.0 / rho))
    assert np.linalg.norm(Lh + Sh - D) / np.linalg.norm(D) < 1e-3
    assert np.linalg.norm(Lh - L0) / np.linalg.norm(L0) < 2e-2
    assert np.linalg.norm(Sh - S0) / np.linalg.norm(S0) < 2e-2
    assert E[-1] < E[10]


def test_cpa_run_tracks_the_exact_run():
    """With enough terms the method's ADMM (FP64 CPA shrinkage) follows the
    exact-SVT run: both are the same iteration up to the shrinkage error."""
    m, n = 40, 32
    L0 = RNG.standard_normal((m, 3)) @ RNG.standard_normal((3, n))
    D = L0 + 0.05 * RNG.standard_normal((m, n))
    rho = m * n / (4.0 * np.abs(D).sum())
    eta = 1.0 / np.sqrt(max(m, n))
    Le, _, _ = A.rpca_admm(D, eta / rho, 30, A.svt_exact(1.0 / rho))
    Lc, _, _ = A.rpca_admm(D, eta / rho, 30, A.svt_cpa(1.0 / rho, 120))
    assert np.linalg.norm(Lc - Le) / np.linalg.norm(Le) < 2e-2


def test_eps_schedule_is_the_papers_piecewise_rule():
    """Eq. recommendation_epsilon: 0.5e-4 above E_l = 0.03, 1.5e-4 down to
    (and excluding) E_m = 6e-4, 0.5e-3 below; E_l itself and E_m itself
    fall in the lower branch of their comparison."""
    assert A.eps_fraction(2.0) == 0.5e-4
    assert A.eps_fraction(0.0300001) == 0.5e-4
    assert A.eps_fraction(0.03) == 1.5e-4
    assert A.eps_fraction(6.0001e-4) == 1.5e-4
    assert A.eps_fraction(6e-4) == 0.5e-3
    assert A.eps_fraction(0.0) == 0.5e-3


def test_lambda_bound_sym_equals_the_gram_bound():
    """On S = X^T X the symmetric-matrix bound is the library's bound of X
    (the C oracle's implementation of the same definition)."""
    X = RNG.standard_normal((30, 12))
    v0 = O.start_vector(0x1705071120000000, 12)
    for iters in (1, 5, 20):
        ref = O.lambda_bound(X, iters, 0.01, v0)["lam"]
        assert abs(A.lambda_bound_sym(X.T @ X, iters, 0.01, v0) - ref) <= 1e-12 * ref


def test_sparse_svt_reduces_to_dense_when_everything_is_kept():
    """With a fraction keeping all p^2 entries and T = Id the sparse step is
    the dense Algorithm 1 with the Gram bound."""
    X = RNG.standard_normal((20, 9))
    f = A.svt_cpa_sparse(0.5, 12, np.eye(9))
    saved = A.eps_fraction
    try:
        A.eps_fraction = lambda E: 1.0
        got = f(X, 1.0)
    finally:
        A.eps_fraction = saved
    lam = O.lambda_bound(X, 20, 0.01, O.start_vector(0x1705071120000000, 9))["lam"]
    assert np.allclose(got, O.cpa(X, O.Shrink(O.SOFT, 0.5), 12, lam), atol=1e-12)
    assert A.kth_largest_abs(np.array([[3.0, -5.0], [1.0, 2.0]]), 2) == 3.0
