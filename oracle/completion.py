"""FP64 reference of the synthetic completion test (test infrastructure only).

Section V, Comparison with Existing Methods restores a corrupted matrix with the inpainting problem of
Section V, Texture Image Inpainting (Eq. texture_repaire4) without its average term.  Its ADMM form
(the appendix ADMM Applicable Forms, Texture Image Inpainting, Eq. admm_algorithm_inp, the z^(5) block dropped with the
average term) works on z = K l with

  K = [Id; Psi; Omega; Id],   Psi the orthonormal 2-D DCT, Omega the
                              observation mask as a diagonal operator,

and one iteration from (z_t, u_t) reads

  l_{t+1} = (K^T K)^{-1} K^T (z_t - u_t)
  z1 = prox_{(1/rho)|.|_*}(l + u1)         singular value shrinkage
  z2 = prox_{(eta/rho)|.|_1}(Psi l + u2)    soft threshold of DCT coefficients
  z3 = Pi_I(Omega l + u3) = Omega i         the observed values
  z4 = Pi_D(l + u4)                         entries clipped to [0, 1]
  u_{t+1} = u_t + K l_{t+1} - z_{t+1}.

Psi^T Psi = Id and Omega^T Omega = Omega, so K^T K = 3 Id + Omega is
diagonal and the least-squares step is l = (a1 + Psi^T a2 + Omega a3 + a4)
/ (3 + omega) with a_i = z_i - u_i.  Start (Section V, Texture Image Inpainting): l_0 = u_0 = all
ones, z_0 = K l_0.  E_t = |l_t - l_{t-1}|_F / |l_t|_F, the quantity Section
IV's footnote names for this very algorithm.

Psi acts on an m x n matrix L as C_m L C_n^T with C_p the orthonormal DCT-II
matrix, C_p[k, j] = s_k cos(pi (2j + 1) k / (2p)), s_0 = sqrt(1/p),
s_k = sqrt(2/p).  The shrinkage step is a callable (exact shrinkage or
Algorithm 1 in FP64, see oracle.admm).
"""
from __future__ import annotations

import numpy as np

from oracle.admm import soft


def dct_matrix(p):
    """Orthonormal DCT-II matrix, written from its definition."""
    k = np.arange(p)[:, None].astype(np.float64)
    j = np.arange(p)[None, :].astype(np.float64)
    s = np.where(k == 0, np.sqrt(1.0 / p), np.sqrt(2.0 / p))
    return s * np.cos(np.pi * (2.0 * j + 1.0) * k / (2.0 * p))


def psi(Lm, Cm, Cn):
    """Psi l: the 2-D DCT coefficients C_m L C_n^T."""
    return Cm @ Lm @ Cn.T


def psi_t(Am, Cm, Cn):
    """Psi^T a: C_m^T A C_n."""
    return Cm.T @ Am @ Cn


def ls_update(a1, a2, a3, a4, omega, Cm, Cn):
    """(K^T K)^{-1} K^T a for a = (a1, a2, a3, a4), written out."""
    return (a1 + psi_t(a2, Cm, Cn) + omega * a3 + a4) / (3.0 + omega)


def completion_admm(I, mask, tau_l1, iters, svt, tol=0.0):
    """Runs the ADMM on the observed matrix I (values where mask == 1).
    Returns (l, z1, E): the last least-squares iterate l, the last
    shrinkage output z1 and the list of E_t."""
    I = np.asarray(I, dtype=np.float64)
    omega = (np.asarray(mask) != 0).astype(np.float64)
    m, n = I.shape
    Cm, Cn = dct_matrix(m), dct_matrix(n)
    z3_fixed = omega * I
    l = np.ones((m, n))
    u1, u2, u3, u4 = (np.ones((m, n)) for _ in range(4))
    z1, z2, z3, z4 = l.copy(), psi(l, Cm, Cn), omega * l, l.copy()
    E = []
    for _ in range(iters):
        l_prev = l
        l = ls_update(z1 - u1, z2 - u2, z3 - u3, z4 - u4, omega, Cm, Cn)
        E.append(float(np.linalg.norm(l - l_prev) / np.linalg.norm(l)))
        P = psi(l, Cm, Cn)
        z1 = svt(l + u1)
        z2 = soft(P + u2, tau_l1)
        z3 = z3_fixed
        z4 = np.clip(l + u4, 0.0, 1.0)
        u1 = u1 + l - z1
        u2 = u2 + P - z2
        u3 = u3 + omega * l - z3
        u4 = u4 + l - z4
        if tol > 0.0 and E[-1] < tol:
            break
    return l, z1, E
