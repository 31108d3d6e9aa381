"""FP64 reference of the background-modelling ADMM (test infrastructure only).

the appendix ADMM Applicable Forms, Background Modeling, Eq. admm_algorithm_mod: min |l|_* + eta |s|_1 subject to
l + s = d, rewritten with z = K l', K = [[I, 0], [0, I], [I, I]] and solved
by ADMM with step rho.  One iteration, from (z_t, u_t):

  l'_{t+1} = (K^T K)^{-1} K^T (z_t - u_t)
  z1 = prox_{(1/rho)|.|_*}(l_{t+1} + u1_t)       (singular value shrinkage)
  z2 = prox_{(eta/rho)|.|_1}(s_{t+1} + u2_t)     (entrywise soft threshold)
  z3 = projection onto {x = d}                   (= d)
  u_{t+1} = u_t + K l'_{t+1} - z_{t+1}

(K^T K)^{-1} = (1/3) [[2, -1], [-1, 2]] and K^T a = (a1 + a3, a2 + a3), so
with a_i = z_i - u_i:  l = (2 a1 - a2 + a3) / 3,  s = (-a1 + 2 a2 + a3) / 3.
Start (Section V, Background Modeling of Video): l_0 = s_0 = u_0 = all ones and
z_0 = K l'_0.  E_t = |l_t - l_{t-1}|_F / |l_t|_F (the stopping quantity of
the stopping-criterion footnote of Section V, Optimization Tools, and Section V, Effects of Thresholding Value).

The shrinkage step is a callable: the exact shrinkage (Jacobi SVD) for the
oracle-SVT run, or Algorithm 1 in FP64 for the method's own run, also with
the sparsity-based reduction and its threshold schedule of Section V, Effects of Thresholding Value
(Eq. recommendation_epsilon): eps = the k-th largest |Phi_ij| with k a
fraction of p^2 chosen from the current E_t.
"""
from __future__ import annotations

import numpy as np

import oracle as O


def soft(x, t):
    """Entrywise soft threshold, the proximal map of t |.|_1."""
    return np.sign(x) * np.maximum(np.abs(x) - t, 0.0)


def ls_update(z1, z2, z3, u1, u2, u3):
    """(K^T K)^{-1} K^T (z - u), written out."""
    a1, a2, a3 = z1 - u1, z2 - u2, z3 - u3
    return (2.0 * a1 - a2 + a3) / 3.0, (-a1 + 2.0 * a2 + a3) / 3.0


def svt_exact(tau):
    s = O.Shrink(O.SOFT, tau)
    return lambda X: O.shrink_exact(X, s)


def svt_cpa(tau, L, iters=20, margin=0.01, seed=0x1705071120000000):
    """Algorithm 1 in FP64 with Lambda_max from the power-iteration bound."""
    s = O.Shrink(O.SOFT, tau)

    def f(X):
        p = min(X.shape)
        lam = O.lambda_bound(X, iters, margin, O.start_vector(seed, p))["lam"]
        return O.cpa(X, s, L, lam)
    return f


E_L, E_M = 0.3e-1, 6e-4   # the schedule's E_l and E_m (Section V, Effects of Thresholding Value)


def eps_fraction(E):
    """Fraction of the p^2 entries of |Phi| kept (k = fraction p^2) for the
    current E_t, Eq. recommendation_epsilon."""
    if E > E_L:
        return 0.5e-4
    if E > E_M:
        return 1.5e-4
    return 0.5e-3


def lambda_bound_sym(S, iters, margin, v0):
    """The power-iteration bound of the library's definition applied to a
    symmetric matrix S (the thresholded Phi_): `iters` normalised steps
    v <- S v / |S v| from v0, theta = v^T S v, r = |S v - theta v|,
    lambda = min((theta + r)(1 + margin), trace S); a non-positive result
    falls back to trace S, or 1."""
    S = np.asarray(S, dtype=np.float64)
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    for _ in range(iters):
        w = S @ v
        nw = np.linalg.norm(w)
        if not nw > 0.0:
            break
        v = w / nw
    w = S @ v
    th = float(v @ w)
    r = float(np.linalg.norm(w - th * v))
    tr = float(np.trace(S))
    lam = min((th + r) * (1.0 + margin), tr)
    if not lam > 0.0:
        lam = tr if tr > 0.0 else 1.0
    return lam


def kth_largest_abs(S, k):
    a = np.sort(np.abs(np.asarray(S, dtype=np.float64)).ravel())[::-1]
    return float(a[min(max(k, 1), a.size) - 1])


def svt_cpa_sparse(tau, L, T, iters=20, margin=0.01, seed=0x1705071120000000):
    """Algorithm 1 with the sparsity-based reduction: Phi = T G T^T, entries
    below eps = K(|Phi|, ceil(frac p^2)) set to zero, Lambda_max the power
    bound of the thresholded Phi_.  Called as svt(X, E) with the current
    E_t choosing frac (eps_fraction)."""
    s = O.Shrink(O.SOFT, tau)

    def f(X, E):
        p = min(X.shape)
        Phi = O.phi(X, T)
        k = int(np.ceil(eps_fraction(E) * p * p))
        eps = kth_largest_abs(Phi, k)
        Phs = np.where(np.abs(Phi) >= eps, Phi, 0.0)
        lam = lambda_bound_sym(Phs, iters, margin, O.start_vector(seed, p))
        return O.cpa(X, s, L, lam, T=T, eps_thr=eps)
    return f


def rpca_admm(D, tau_l1, iters, svt, tol=0.0, schedule=False):
    """Runs the ADMM; returns (z1, z2, E) with z1 the low-rank part (the
    shrinkage output), z2 the sparse part and E the list of E_t.  With
    `schedule`, svt is called as svt(X, E_t)."""
    D = np.asarray(D, dtype=np.float64)
    ones = np.ones_like(D)
    l, s = ones.copy(), ones.copy()
    u1, u2, u3 = ones.copy(), ones.copy(), ones.copy()
    z1, z2, z3 = l.copy(), s.copy(), l + s
    E = []
    for _ in range(iters):
        l_prev = l
        l, s = ls_update(z1, z2, z3, u1, u2, u3)
        E.append(float(np.linalg.norm(l - l_prev) / np.linalg.norm(l)))
        z1 = svt(l + u1, E[-1]) if schedule else svt(l + u1)
        z2 = soft(s + u2, tau_l1)
        z3 = D
        u1 = u1 + l - z1
        u2 = u2 + s - z2
        u3 = u3 + l + s - z3
        if tol > 0.0 and E[-1] < tol:
            break
    return z1, z2, E
