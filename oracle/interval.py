"""FP64 reference of the guarded series interval for a thresholded Phi
(test infrastructure only).

Section III-B builds the filter on [0, Lambda_max].  After the entry
threshold of Eq. threshold_components, Phi_ = Phi - E (E the removed
entries) is still symmetric but in general no longer PSD, and its negative
eigenvalues fall outside the series' interval, where T_k grows.  The library
keeps the interval as written (reading R8); the guarded form studied here
moves the lower end to a = -|E|_F.  Weyl's inequality and Phi being PSD give
lambda_min(Phi_) >= lambda_min(Phi) - |E|_2 >= -|E|_F, so [a, b] with
b = Lambda_max holds the whole spectrum of Phi_:

  c_k = (2/L) sum_{l=1}^{L} cos(k theta_l) h(a + (b - a)(cos theta_l + 1)/2),
        theta_l = pi (l - 1/2) / L                 (Eq. chebychev_coeff_shifted
                                                     with [0, lambda] -> [a, b])
  B = (2 Phi_ - (a + b) Id) / (b - a)
  H = c_0/2 Id + sum_{k=1}^{L-1} c_k T_k(B)        (forward recurrence, Algorithm 1)
  Y = X T^T H T  (m >= n),  T^T H T X  (m < n)     (Eq. SVD_fil)

h(x) is 0 for x <= 0 (no singular value lies there).  With a = 0 and no
threshold this is Algorithm 1 itself.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O


def removed_norm(Phi, eps):
    """|E|_F for E the entries of Phi with |Phi_ij| < eps."""
    Phi = np.asarray(Phi, dtype=np.float64)
    E = np.where(np.abs(Phi) >= eps, 0.0, Phi)
    return float(np.linalg.norm(E))


def threshold(Phi, eps):
    """Phi_: the entries with |Phi_ij| >= eps kept, the rest zero."""
    Phi = np.asarray(Phi, dtype=np.float64)
    return np.where(np.abs(Phi) >= eps, Phi, 0.0)


def coeffs_interval(s, L, a, b):
    """c_k, k = 0..L-1, of h on [a, b] (plain loops)."""
    c = np.zeros(L)
    for k in range(L):
        acc = 0.0
        for l in range(1, L + 1):
            th = math.pi * (l - 0.5) / L
            x = a + 0.5 * (b - a) * (math.cos(th) + 1.0)
            acc += math.cos(k * th) * (O.h(s, x) if x > 0.0 else 0.0)
        c[k] = 2.0 / L * acc
    return c


def filter_matrix(S, c, a, b):
    """H = c_0/2 Id + sum_{k>=1} c_k T_k(B), B = (2 S - (a+b) Id)/(b - a),
    by the forward three-term recurrence."""
    p = S.shape[0]
    Id = np.eye(p)
    B = (2.0 * S - (a + b) * Id) / (b - a)
    H = 0.5 * c[0] * Id
    if len(c) == 1:
        return H
    Z0, Z1 = Id, B
    H = H + c[1] * Z1
    for k in range(2, len(c)):
        Z0, Z1 = Z1, 2.0 * B @ Z1 - Z0
        H = H + c[k] * Z1
    return H


def cpa_interval(X, s, L, a, b, T=None, eps_thr=-1.0, return_H=False):
    """Algorithm 1 with the transform T, the entry threshold eps_thr (< 0:
    none) and the series on [a, b]."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    tall = m >= n
    G = X.T @ X if tall else X @ X.T
    p = G.shape[0]
    Tm = np.eye(p) if T is None else np.asarray(T, dtype=np.float64)
    Phi = Tm @ G @ Tm.T
    if eps_thr >= 0.0:
        Phi = threshold(Phi, eps_thr)
    H = filter_matrix(Phi, coeffs_interval(s, L, a, b), a, b)
    F = Tm.T @ H @ Tm
    Y = X @ F if tall else F @ X
    return (Y, H) if return_H else Y


def guarded_cpa(X, s, L, lam, T, eps_thr, return_H=False):
    """The guarded form: a = -|Phi - Phi_|_F, b = lam."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    G = X.T @ X if m >= n else X @ X.T
    Phi = T @ G @ T.T
    a = -removed_norm(Phi, eps_thr)
    return cpa_interval(X, s, L, a, lam, T, eps_thr, return_H)
