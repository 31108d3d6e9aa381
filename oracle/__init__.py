"""FP64 CPU oracle for CPA singular value shrinkage (arXiv 1705.07112).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product library never does.  It
shares no code with the CUDA path.  The arithmetic lives in plain C
(``cpa_oracle.c``, FP64, plain loops in the paper's order); this module only
compiles it with gcc and marshals numpy arrays.

Functions and the passage each follows:

* ``h`` / ``g``           shrinkage responses, Eq. filter_response_ours
* ``coeffs``              shifted Chebyshev coefficients, Eq. chebychev_coeff_shifted
* ``coeffs_from_nodes``   unshifted coefficients, Eq. chebychev_coeff_discrete
* ``series_cos`` / ``series_rec``  truncated series, Eqs. chebychev_series,
                          chebychev_polynomial and chebyche2
* ``gram``                Gram matrix of the smaller side (Algorithm 1, T = Id)
* ``phi``                 T G T^T (Eq. sing_shrink_exact_sparse), no threshold
* ``cpa``                 Algorithm 1, dense, optional transform T and entry
                          threshold (Eqs. sing_shrink_exact_sparse,
                          threshold_components, recurrence_our_method, SVD_fil)
* ``cpa_clenshaw``        the same filter summed by Clenshaw's recurrence
* ``cpa_vec``             the same filter applied to one vector
                          (Eq. prop_another_form), for sampled outputs at any size
* ``cpa_block`` / ``filter_block``  the same vector form on a block of vectors
                          at once (numpy's matmul as the product primitive),
                          with the Gram matrix given through X or as a symmetric
                          matrix S (a thresholded Phi)
* ``lambda_bound``        power-iteration bound on Lambda_max (the paper names no
                          method; reading stated in the C source)
* ``svd_jacobi``          one-sided Jacobi SVD
* ``eig_jacobi``          cyclic Jacobi symmetric eigendecomposition
* ``shrink_exact``        exact shrinkage via SVD, Eq. sing_shrink_exact
* ``shrink_exact_evd``    exact shrinkage via EVD, Eq. sing_shrink_exact_from_eig2
* ``start_vector``        SplitMix64 start vector for the power iteration
* ``singular_values``     singular values through LAPACK (a library primitive,
                          for spectra of large matrices)
* ``shrink_exact_lapack`` exact shrinkage U diag(g(sigma)) V^T (Eq.
                          sing_shrink_exact) with LAPACK's SVD as the
                          decomposition step, for judging results at large sizes
* ``spectral_errors``     |G_hat(X) - G(X)|_F / |G(X)|_F of the FP64 CPA for many
                          orders at once from the singular values (the
                          spectral error identity)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HARD, SOFT, WSOFT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpa_oracle.c")
_LIB = os.path.join(_HERE, "liborc_cpa.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle's C source into a shared library (gcc, -O2, FP64,
    no fast-math so IEEE rounding is kept)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_h": (_d, [_i, _d, _d, _d, _d, _d]),
                "orc_g": (_d, [_i, _d, _d, _d, _d, _d]),
                "orc_coeffs": (None, [_i, _d, _d, _d, _d, _i, _d, _P]),
                "orc_coeffs_from_nodes": (None, [_i, _P, _P]),
                "orc_series_cos": (_d, [_P, _i, _d]),
                "orc_series_rec": (_d, [_P, _i, _d]),
                "orc_cheb_T": (_d, [_i, _d]),
                "orc_gram": (None, [_P, _i, _i, _P]),
                "orc_phi": (None, [_P, _i, _i, _P, _P]),
                "orc_cpa": (_i, [_P, _i, _i, _i, _d, _d, _d, _d, _i, _d, _P, _d, _P, _P]),
                "orc_cpa_clenshaw": (_i, [_P, _i, _i, _i, _d, _d, _d, _d, _i, _d, _P, _d, _P, _P]),
                "orc_cpa_vec": (_i, [_P, _i, _i, _i, _d, _d, _d, _d, _i, _d, _P, _P]),
                "orc_lambda_bound": (_i, [_P, _i, _i, _i, _d, _P, _P]),
                "orc_svd_jacobi": (_i, [_P, _i, _i, _P, _P, _P, _d, _i]),
                "orc_eig_jacobi": (_i, [_P, _i, _P, _P, _d, _i]),
                "orc_shrink_exact": (_i, [_P, _i, _i, _i, _d, _d, _d, _d, _P, _P]),
                "orc_shrink_exact_evd": (_i, [_P, _i, _i, _i, _d, _d, _d, _d, _P]),
                "orc_start_vector": (None, [ctypes.c_uint64, _i, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


def _p(a):
    return a.ctypes.data_as(_P) if a is not None else None


class Shrink:
    """Parameters of the shrinkage response (Eq. filter_response_ours).

    kind: HARD (W = 0), SOFT (W = tau), WSOFT (W = w(x) = c/(sqrt(max(x-noise,0))+eps));
    tau: threshold on sigma for HARD/SOFT.
    """

    def __init__(self, kind=SOFT, tau=0.0, c=0.0, eps=1e-8, noise=0.0):
        self.kind, self.tau, self.c, self.eps, self.noise = int(kind), float(tau), float(c), float(eps), float(noise)

    def args(self):
        return (self.kind, self.tau, self.c, self.eps, self.noise)

    def __repr__(self):
        return "Shrink(kind=%d, tau=%g, c=%g, eps=%g, noise=%g)" % self.args()


def h(s: Shrink, x: float) -> float:
    return _load().orc_h(*s.args(), float(x))


def g(s: Shrink, sigma: float) -> float:
    return _load().orc_g(*s.args(), float(sigma))


def coeffs(s: Shrink, alpha: int, lam: float) -> np.ndarray:
    out = np.zeros(alpha)
    _load().orc_coeffs(*s.args(), int(alpha), float(lam), _p(out))
    return out


def coeffs_from_nodes(hs) -> np.ndarray:
    hs = _arr(hs)
    out = np.zeros(hs.size)
    _load().orc_coeffs_from_nodes(hs.size, _p(hs), _p(out))
    return out


def series_cos(ck, x: float) -> float:
    ck = _arr(ck)
    return _load().orc_series_cos(_p(ck), ck.size, float(x))


def series_rec(ck, x: float) -> float:
    ck = _arr(ck)
    return _load().orc_series_rec(_p(ck), ck.size, float(x))


def cheb_T(k: int, x: float) -> float:
    return _load().orc_cheb_T(int(k), float(x))


def gram(X) -> np.ndarray:
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    G = np.zeros((p, p))
    _load().orc_gram(_p(X), m, n, _p(G))
    return G


def phi(X, T=None) -> np.ndarray:
    """Phi = T G T^T before thresholding (Eq. sing_shrink_exact_sparse)."""
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    Tm = _arr(T, (p, p)) if T is not None else None
    out = np.zeros((p, p))
    _load().orc_phi(_p(X), m, n, _p(Tm), _p(out))
    return out


def cpa(X, s: Shrink, alpha: int, lam: float, T=None, eps_thr: float = -1.0,
        return_H: bool = False):
    """Algorithm 1 in FP64 (dense).  Returns Y (and H_hat if asked)."""
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    Tm = _arr(T, (p, p)) if T is not None else None
    Y = np.zeros((m, n))
    H = np.zeros((p, p)) if return_H else None
    rc = _load().orc_cpa(_p(X), m, n, *s.args(), int(alpha), float(lam), _p(Tm),
                         float(eps_thr), _p(Y), _p(H))
    if rc:
        raise ValueError("orc_cpa: invalid arguments (alpha=%r, lam=%r)" % (alpha, lam))
    return (Y, H) if return_H else Y


def cpa_clenshaw(X, s: Shrink, alpha: int, lam: float, T=None, eps_thr: float = -1.0,
                 return_H: bool = False):
    """Algorithm 1 with the filter summed by Clenshaw's recurrence (FP64)."""
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    Tm = _arr(T, (p, p)) if T is not None else None
    Y = np.zeros((m, n))
    H = np.zeros((p, p)) if return_H else None
    rc = _load().orc_cpa_clenshaw(_p(X), m, n, *s.args(), int(alpha), float(lam), _p(Tm),
                                  float(eps_thr), _p(Y), _p(H))
    if rc:
        raise ValueError("orc_cpa_clenshaw: invalid arguments (alpha=%r, lam=%r)" % (alpha, lam))
    return (Y, H) if return_H else Y


def cpa_vec(X, s: Shrink, alpha: int, lam: float, v) -> np.ndarray:
    """H_hat(G) v with G the Gram matrix of the smaller side of X."""
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    v = _arr(v, (p,))
    out = np.zeros(p)
    rc = _load().orc_cpa_vec(_p(X), m, n, *s.args(), int(alpha), float(lam), _p(v), _p(out))
    if rc:
        raise ValueError("orc_cpa_vec: invalid arguments")
    return out


def lambda_bound(X, iters: int, margin: float, v0) -> dict:
    X = _arr(X)
    m, n = X.shape
    p = min(m, n)
    v0 = _arr(v0, (p,))
    out = np.zeros(4)
    rc = _load().orc_lambda_bound(_p(X), m, n, int(iters), float(margin), _p(v0), _p(out))
    if rc:
        raise ValueError("orc_lambda_bound: zero start vector")
    return {"theta": out[0], "resid": out[1], "trace": out[2], "lam": out[3]}


def svd_jacobi(X, tol=1e-15, max_sweeps=60):
    """One-sided Jacobi SVD of a tall X: returns (W = X V, V, s), columns of W
    are sigma_i u_i."""
    X = _arr(X)
    m, n = X.shape
    W = np.zeros((m, n))
    V = np.zeros((n, n))
    s = np.zeros(n)
    sw = _load().orc_svd_jacobi(_p(X), m, n, _p(W), _p(V), _p(s), float(tol), int(max_sweeps))
    if sw < 0:
        raise RuntimeError("orc_svd_jacobi: %s" % ("m < n" if sw == -2 else "no convergence"))
    return W, V, s


def eig_jacobi(S, tol=1e-15, max_sweeps=60):
    S = _arr(S)
    p = S.shape[0]
    w = np.zeros(p)
    V = np.zeros((p, p))
    sw = _load().orc_eig_jacobi(_p(S), p, _p(w), _p(V), float(tol), int(max_sweeps))
    if sw < 0:
        raise RuntimeError("orc_eig_jacobi: no convergence")
    return w, V


def shrink_exact(X, s: Shrink, return_sv: bool = False):
    X = _arr(X)
    m, n = X.shape
    Y = np.zeros((m, n))
    sv = np.zeros(min(m, n))
    rc = _load().orc_shrink_exact(_p(X), m, n, *s.args(), _p(Y), _p(sv))
    if rc:
        raise RuntimeError("orc_shrink_exact: Jacobi SVD did not converge")
    return (Y, sv) if return_sv else Y


def shrink_exact_evd(X, s: Shrink):
    X = _arr(X)
    m, n = X.shape
    Y = np.zeros((m, n))
    rc = _load().orc_shrink_exact_evd(_p(X), m, n, *s.args(), _p(Y))
    if rc:
        raise RuntimeError("orc_shrink_exact_evd: Jacobi EVD did not converge")
    return Y


def start_vector(seed: int, p: int) -> np.ndarray:
    out = np.zeros(p)
    _load().orc_start_vector(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(p), _p(out))
    return out


def approx_error_spectral(sv, s: Shrink, alpha: int, lam: float) -> float:
    """|G_hat(X) - G(X)|_F for the FP64 CPA, from the singular values alone.

    X H_hat(X^T X) and the exact shrinkage share singular vectors (Eq. ATA_eig_fil
    with T = Id), so the difference has singular values
    sigma_i |h_hat(sigma_i^2) - h(sigma_i^2)|.  h_hat is the shifted series of
    Eq. chebychev_series_matrix_shift2 evaluated at 2 sigma^2/lam - 1.
    """
    ck = coeffs(s, alpha, lam)
    tot = 0.0
    for sig in np.asarray(sv, dtype=np.float64):
        x = sig * sig
        xh = 2.0 * x / lam - 1.0
        hh = series_rec(ck, xh)
        tot += (sig * (hh - h(s, x))) ** 2
    return float(np.sqrt(tot))


def _series_block(prod, s: Shrink, alpha: int, lam: float, V) -> np.ndarray:
    """H_hat V for the shifted series of Algorithm 1 (Eqs.
    chebychev_series_matrix_shift2 and recurrence_our_method applied to the
    columns of V, as Eq. prop_another_form applies it to one vector):
    Z_0 = V, Z_1 = B_hat V, Z_k = 2 B_hat Z_{k-1} - Z_{k-2}, B_hat Z =
    (2/lam) prod(Z) - Z, H_hat V = c_0/2 Z_0 + sum_{k>=1} c_k Z_k.
    prod(Z) is the product of the symmetric matrix with Z."""
    if alpha < 1 or not (lam > 0.0):
        raise ValueError("series: invalid arguments (alpha=%r, lam=%r)" % (alpha, lam))
    c = coeffs(s, alpha, lam)
    V = np.asarray(V, dtype=np.float64)
    z0 = V
    out = 0.5 * c[0] * z0
    if alpha == 1:
        return out
    z1 = 2.0 / lam * prod(z0) - z0
    out = out + c[1] * z1
    for k in range(2, alpha):
        z2 = 2.0 * (2.0 / lam * prod(z1) - z1) - z0
        out = out + c[k] * z2
        z0, z1 = z1, z2
    return out


def cpa_block(X, s: Shrink, alpha: int, lam: float, V) -> np.ndarray:
    """H_hat(G) V, G the Gram matrix of the smaller side of X, for the p x k
    block V (p = min(m, n)); G Z is formed as X^T (X Z) or X (X^T Z)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    V = np.asarray(V, dtype=np.float64)
    if V.shape[0] != min(m, n):
        raise ValueError("cpa_block: V must have min(m, n) rows")
    prod = (lambda Z: X.T @ (X @ Z)) if m >= n else (lambda Z: X @ (X.T @ Z))
    return _series_block(prod, s, alpha, lam, V)


def filter_block(S, s: Shrink, alpha: int, lam: float, V) -> np.ndarray:
    """H_hat(S) V for a symmetric p x p matrix S given explicitly (the
    thresholded Phi of Eq. threshold_components), p x k block V."""
    S = np.asarray(S, dtype=np.float64)
    return _series_block(lambda Z: S @ Z, s, alpha, lam, V)


def singular_values(X) -> np.ndarray:
    """Singular values of X in descending order, LAPACK's SVD (gesdd)."""
    return np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)


def shrink_exact_lapack(X, s: Shrink) -> np.ndarray:
    """U diag(g(sigma_i)) V^T (Eq. sing_shrink_exact), the thin SVD from
    LAPACK, g from the scalar response of Eq. filter_response_ours."""
    X = np.asarray(X, dtype=np.float64)
    U, sv, Vt = np.linalg.svd(X, full_matrices=False)
    gs = np.array([g(s, x) for x in sv])
    return (U * gs) @ Vt


def spectral_errors(sv, s: Shrink, lam: float, alphas) -> np.ndarray:
    """Relative Frobenius error of the FP64 CPA against the exact shrinkage
    for every alpha in `alphas`, from the singular values alone: X H_hat(X^T X)
    and the exact shrinkage share singular vectors, so the difference has
    singular values sigma_i |h_hat(sigma_i^2) - h(sigma_i^2)| (as in
    approx_error_spectral).  When the exact shrinkage is 0 the error is
    relative to |X|_F."""
    sv = np.asarray(sv, dtype=np.float64)
    x = sv * sv
    hx = np.array([h(s, v) for v in x])
    exact = float(np.sqrt(np.sum((sv * hx) ** 2)))
    den = exact if exact > 0 else float(np.sqrt(np.sum(x)))
    t = 2.0 * x / lam - 1.0
    out = []
    for alpha in alphas:
        ck = coeffs(s, int(alpha), lam)
        # the shifted series at t by the three-term recurrence (Eq. chebyche2)
        z0, z1 = np.ones_like(t), t
        hh = 0.5 * ck[0] * z0 + (ck[1] * z1 if alpha > 1 else 0.0)
        for k in range(2, int(alpha)):
            z0, z1 = z1, 2.0 * t * z1 - z0
            hh = hh + ck[k] * z1
        out.append(float(np.sqrt(np.sum((sv * (hh - hx)) ** 2))) / den)
    return np.array(out)
