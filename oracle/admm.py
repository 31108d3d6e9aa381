"""FP64 reference of the background-modelling ADMM (test infrastructure only).

Appendix B, Eq. admm_algorithm_mod: min |l|_* + eta |s|_1 subject to
l + s = d, rewritten with z = K l', K = [[I, 0], [0, I], [I, I]] and solved
by ADMM with step rho.  One iteration, from (z_t, u_t):

  l'_{t+1} = (K^T K)^{-1} K^T (z_t - u_t)
  z1 = prox_{(1/rho)|.|_*}(l_{t+1} + u1_t)       (singular value shrinkage)
  z2 = prox_{(eta/rho)|.|_1}(s_{t+1} + u2_t)     (entrywise soft threshold)
  z3 = projection onto {x = d}                   (= d)
  u_{t+1} = u_t + K l'_{t+1} - z_{t+1}

(K^T K)^{-1} = (1/3) [[2, -1], [-1, 2]] and K^T a = (a1 + a3, a2 + a3), so
with a_i = z_i - u_i:  l = (2 a1 - a2 + a3) / 3,  s = (-a1 + 2 a2 + a3) / 3.
Start (Section V-C, background modelling): l_0 = s_0 = u_0 = all ones and
z_0 = K l'_0.  E_t = |l_t - l_{t-1}|_F / |l_t|_F (the stopping quantity of
Section IV's footnote and Section V-D).

The shrinkage step is a callable: the exact shrinkage (Jacobi SVD) for the
oracle-SVT run, or Algorithm 1 in FP64 for the method's own run.
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


def rpca_admm(D, tau_l1, iters, svt, tol=0.0):
    """Runs the ADMM; returns (z1, z2, E) with z1 the low-rank part (the
    shrinkage output), z2 the sparse part and E the list of E_t."""
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
        z1 = svt(l + u1)
        z2 = soft(s + u2, tau_l1)
        z3 = D
        u1 = u1 + l - z1
        u2 = u2 + s - z2
        u3 = u3 + l + s - z3
        if tol > 0.0 and E[-1] < tol:
            break
    return z1, z2, E
