"""ctypes binding of libcpa (include/cpa.h).  Argument marshalling only: every
step of the shrinkage runs in the library's CUDA kernels.  PyTorch provides
device memory and the current stream.  There is no CPU fallback: if the
library is missing or cannot load, every call raises."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpa.so")

CPA_OK, CPA_ERR_INVALID_ARG, CPA_ERR_CUDA, CPA_ERR_NO_MEMORY = 0, 1, 2, 3
CPA_ERR_NONFINITE, CPA_ERR_BOUND, CPA_ERR_TIMEOUT, CPA_ERR_UNSUPPORTED = 4, 5, 6, 7
HARD, SOFT, WSOFT = 0, 1, 2
FP32, TF32, BF16, BF16X3 = 0, 1, 2, 3
PREC = {"fp32": FP32, "tf32": TF32, "bf16": BF16, "bf16x3": BF16X3}

# every function include/cpa.h declares
EXPORTS = ["cpa_create", "cpa_destroy", "cpa_status_string", "cpa_last_error", "cpa_coeffs",
           "cpa_lambda_bound", "cpa_svt", "cpa_svt_host", "cpa_get_lambda", "cpa_get_coeffs", "cpa_batch_create",
           "cpa_batch_destroy", "cpa_svt_batched_plan", "cpa_svt_batched", "cpa_batch_lambdas", "cpa_profile_enable",
           "cpa_profile_read", "cpa_kernel_gemm_bf16", "cpa_kernel_split_bf16", "cpa_kernel_topk_eps", "cpa_batch_read_lambdas",
           "cpa_lambda_bound_noalloc", "cpa_mlp_create", "cpa_mlp_destroy", "cpa_mlp_param_count",
           "cpa_mlp_set_params", "cpa_mlp_get_params", "cpa_mlp_forward", "cpa_mlp_gradients",
           "cpa_mlp_train_step", "cpa_batch_features", "cpa_svt_batched_learned", "cpa_batch_read_choices",
           "cpa_admm_create", "cpa_admm_destroy", "cpa_admm_rpca", "cpa_set_option",
           "cpa_completion_create", "cpa_completion_destroy", "cpa_completion_run", "cpa_sync_status",
           "cpa_svt_learned", "cpa_get_order", "cpa_learn_features", "cpa_serve_learned", "cpa_serve_read",
           "cpa_batch_set_config", "cpa_batch_get_config", "cpa_batch_tune"]
BATCH_MMA_SYNC, BATCH_TCGEN05 = 0, 1
ORDER_SIZE, ORDER_GIVEN = 0, 1
OPT_SERIES, SERIES_FORWARD, SERIES_CLENSHAW = 1, 0, 1
OPT_WAIT_KCYCLES, OPT_STALL_TEST, OPT_SPARSE_SKIP, OPT_STREAMS, OPT_MEMBER_SMS, OPT_SPARSE_COMPACT = 2, 3, 4, 5, 6, 7
STAGES = ["prep", "gram", "bound", "coeff", "shift", "recur", "apply", "sparse"]
T_IDENTITY, T_HAAR1_LOWPASS, T_BLOCK_DCT8, T_DCT = 0, 1, 2, 3
SPARSE_OFF, SPARSE_ABS, SPARSE_TOPK = 0, 1, 2


class CpaShrink(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("tau", ctypes.c_double), ("c", ctypes.c_double),
                ("eps", ctypes.c_double), ("noise", ctypes.c_double)]


class CpaSparsify(ctypes.Structure):
    _fields_ = [("transform", ctypes.c_int), ("mode", ctypes.c_int), ("eps_or_frac", ctypes.c_double),
                ("interval", ctypes.c_int)]


class CpaLearnRule(ctypes.Structure):
    _fields_ = [("L_scale", ctypes.c_double), ("margin", ctypes.c_double), ("L_min", ctypes.c_int),
                ("L_max", ctypes.c_int), ("L_fallback", ctypes.c_int), ("use_lambda", ctypes.c_int)]


class CpaError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, _status_string(status), _last_error()))


_lib = None
_lock = threading.Lock()
_vp, _i64, _i32, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_P = ctypes.POINTER


def load(path: str = LIB_PATH):
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libcpa.so not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        sig = {
            "cpa_create": (ctypes.c_int, [_P(_vp), ctypes.c_int]),
            "cpa_destroy": (ctypes.c_int, [_vp]),
            "cpa_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "cpa_last_error": (ctypes.c_char_p, []),
            "cpa_coeffs": (ctypes.c_int, [_P(CpaShrink), ctypes.c_int, _d, _P(_d)]),
            "cpa_lambda_bound": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, ctypes.c_int, _P(_d), _vp]),
            "cpa_svt": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _P(CpaShrink), ctypes.c_int, _d,
                                       ctypes.c_int, _P(CpaSparsify), _vp, _i64, _vp]),
            "cpa_svt_host": (ctypes.c_int, [_vp, ctypes.c_int, _P(_vp), _i64, _i64, _i64, _P(CpaShrink),
                                            ctypes.c_int, _d, ctypes.c_int, _P(CpaSparsify), _P(_vp), _i64, _vp]),
            "cpa_get_lambda": (ctypes.c_int, [_vp, _P(_d), _vp]),
            "cpa_sync_status": (ctypes.c_int, [_vp, _vp]),
            "cpa_batch_set_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "cpa_batch_get_config": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int)]),
            "cpa_batch_tune": (ctypes.c_int, [_vp, _vp, _vp, _P(CpaShrink), ctypes.c_int, ctypes.c_int, _vp,
                                              ctypes.c_int, _P(ctypes.c_int), _P(_d), _vp]),
            "cpa_svt_learned": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _P(CpaShrink), _P(CpaLearnRule),
                                               ctypes.c_int, _vp, _i64, _vp]),
            "cpa_get_order": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int), _vp]),
            "cpa_svt_batched": (ctypes.c_int, [_vp, ctypes.c_int, _P(_vp), _P(_i64), _P(_i64), _P(_i64),
                                               _P(CpaShrink), ctypes.c_int, _P(ctypes.c_int), ctypes.c_int,
                                               _P(_d), ctypes.c_int, _P(_vp), _P(_i64), _vp]),
            "cpa_serve_learned": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _P(_vp), _P(_i64), _P(_i64), _P(_i64),
                                                 _P(CpaShrink), ctypes.c_int, _P(CpaLearnRule), ctypes.c_int,
                                                 _P(_vp), _P(_i64), _vp]),
            "cpa_serve_read": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_int), _P(_d), _P(ctypes.c_int), _vp]),
            "cpa_learn_features": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _P(CpaShrink), _vp, _vp, _vp]),
            "cpa_get_coeffs": (ctypes.c_int, [_vp, _P(_d), ctypes.c_int, _vp]),
            "cpa_batch_create": (ctypes.c_int, [_vp, ctypes.c_int, _P(_i64), _P(_i32), _P(_i32), _P(_i32),
                                                ctypes.c_int, _P(_vp)]),
            "cpa_batch_destroy": (ctypes.c_int, [_vp]),
            "cpa_svt_batched_plan": (ctypes.c_int, [_vp, _vp, _vp, _P(CpaShrink), ctypes.c_int, _vp, ctypes.c_int,
                                               ctypes.c_int, _vp, _vp]),
            "cpa_batch_lambdas": (_vp, [_vp]),
            "cpa_batch_read_lambdas": (ctypes.c_int, [_vp, _P(_d), _vp]),
            "cpa_lambda_bound_noalloc": (ctypes.c_int, [_vp, _i64, _i64, _i64, ctypes.c_int, _P(_d), _vp]),
            "cpa_mlp_create": (ctypes.c_int, [_P(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_uint64]),
            "cpa_mlp_destroy": (ctypes.c_int, [_vp]),
            "cpa_batch_features": (ctypes.c_int, [_vp, _vp, _vp, _P(CpaShrink), ctypes.c_int, _vp, _vp, _vp]),
            "cpa_svt_batched_learned": (ctypes.c_int, [_vp, _vp, _vp, _vp, _P(CpaShrink), ctypes.c_int, _d,
                                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _d,
                                                       ctypes.c_int, _vp, _vp]),
            "cpa_batch_read_choices": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int), _vp]),
            "cpa_mlp_param_count": (_i64, [_vp]),
            "cpa_mlp_set_params": (ctypes.c_int, [_vp, _P(ctypes.c_float), _i64]),
            "cpa_mlp_get_params": (ctypes.c_int, [_vp, _P(ctypes.c_float), _i64]),
            "cpa_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
            "cpa_mlp_gradients": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _P(ctypes.c_float), _i64,
                                                 _P(ctypes.c_float), _vp]),
            "cpa_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                                  _P(ctypes.c_float), _vp]),
            "cpa_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
            "cpa_kernel_gemm_bf16": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _i64, _vp,
                                                    _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_float, _vp,
                                                    ctypes.c_float, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp,
                                                    ctypes.c_int, _vp, _i64, _vp, _vp, _i64, _vp]),
            "cpa_kernel_split_bf16": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, ctypes.c_int, _vp,
                                                     _vp, _i64, _vp]),
            "cpa_kernel_topk_eps": (ctypes.c_int, [_vp, ctypes.c_int, _i64, ctypes.c_longlong, _P(ctypes.c_float),
                                                   _vp]),
            "cpa_profile_read": (ctypes.c_int, [_vp, _P(_d), _P(_i64), ctypes.c_int]),
            "cpa_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
            "cpa_admm_create": (ctypes.c_int, [_vp, _i64, _i64, _P(_vp)]),
            "cpa_admm_destroy": (ctypes.c_int, [_vp]),
            "cpa_admm_rpca": (ctypes.c_int, [_vp, _vp, _i64, _d, _d, ctypes.c_int, ctypes.c_int,
                                             _P(CpaSparsify), ctypes.c_int, ctypes.c_int, _d, _vp, _vp,
                                             _P(ctypes.c_int), _P(_d), _vp]),
            "cpa_completion_create": (ctypes.c_int, [_vp, _i64, _i64, _P(_vp)]),
            "cpa_completion_destroy": (ctypes.c_int, [_vp]),
            "cpa_completion_run": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _d, _d, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _d, _vp, _i64, _vp, _P(ctypes.c_int), _P(_d),
                                                  _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _status_string(s):
    try:
        return load().cpa_status_string(int(s)).decode()
    except Exception:
        return "status %d" % s


def _last_error():
    try:
        return load().cpa_last_error().decode()
    except Exception:
        return ""


def _check(status, where):
    if status != CPA_OK:
        raise CpaError(status, where)


def shrink_struct(kind=SOFT, tau=0.0, c=0.0, eps=1e-8, noise=0.0) -> CpaShrink:
    return CpaShrink(int(kind), float(tau), float(c), float(eps), float(noise))


def _as_shrink(s) -> CpaShrink:
    if isinstance(s, CpaShrink):
        return s
    if isinstance(s, dict):
        return shrink_struct(**s)
    # dataclass-like (inputs.ShrinkSpec)
    return shrink_struct(s.kind, s.tau, s.c, s.eps, s.noise)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _matrix(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2:
        raise ValueError("%s must be a 2-D float32 CUDA tensor" % name)
    if t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError("%s must be row-major with unit column stride" % name)
    return t.data_ptr(), t.shape[0], t.shape[1], t.stride(0)


class Handle:
    """Owns a cpa_handle (device workspace) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.cpa_create(ctypes.byref(h), int(device)), "cpa_create")
        self.ptr = h
        self.device = device

    def close(self):
        if self.ptr:
            self._lib.cpa_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cpa_coeffs(shrink, L: int, lambda_max: float) -> np.ndarray:
    out = np.zeros(int(L), dtype=np.float64)
    s = _as_shrink(shrink)
    _check(load().cpa_coeffs(ctypes.byref(s), int(L), float(lambda_max),
                             out.ctypes.data_as(_P(_d))), "cpa_coeffs")
    return out


def cpa_lambda_bound(h: Handle, X, iters: int = 20, stream=None) -> float:
    ptr, m, n, ld = _matrix(X, "X")
    out = ctypes.c_double()
    _check(load().cpa_lambda_bound(h.ptr, ctypes.c_void_p(ptr), m, n, ld, int(iters), ctypes.byref(out),
                                   _stream_ptr(stream)), "cpa_lambda_bound")
    return out.value


def cpa_lambda_bound_noalloc(X, iters: int = 20, stream=None) -> float:
    """The Lambda_max bound of cpa_lambda_bound computed without a handle
    and without allocating device memory (fixed scratch array inside the
    library; min(m, n) <= 512), for callers that must not allocate."""
    ptr, m, n, ld = _matrix(X, "X")
    out = ctypes.c_double()
    _check(load().cpa_lambda_bound_noalloc(ctypes.c_void_p(ptr), m, n, ld, int(iters), ctypes.byref(out),
                                           _stream_ptr(stream)), "cpa_lambda_bound_noalloc")
    return out.value


def cpa_svt(h: Handle, X, shrink, L: int, lambda_max: float = 0.0, prec="fp32", sparsify=None, Y=None,
            stream=None):
    """CPA singular value shrinkage of X (Algorithm 1).  Returns Y (allocated
    with torch if not given).  lambda_max <= 0: computed on the device."""
    import torch
    ptr, m, n, ld = _matrix(X, "X")
    if Y is None:
        Y = torch.empty((m, n), dtype=torch.float32, device=X.device)
    yptr, ym, yn, ldy = _matrix(Y, "Y")
    if (ym, yn) != (m, n):
        raise ValueError("Y shape mismatch")
    s = _as_shrink(shrink)
    sp = None
    if sparsify is not None:
        sp = ctypes.byref(CpaSparsify(int(sparsify[0]), int(sparsify[1]), float(sparsify[2]),
                                              int(sparsify[3]) if len(sparsify) > 3 else 0))
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt(h.ptr, ctypes.c_void_p(ptr), m, n, ld, ctypes.byref(s), int(L), float(lambda_max), p,
                          sp, ctypes.c_void_p(yptr), ldy, _stream_ptr(stream)), "cpa_svt")
    return Y


def cpa_svt_host(h: Handle, Xs, shrink, L: int, lambda_max: float = 0.0, prec="fp32", sparsify=None, Ys=None,
                 stream=None):
    """cpa_svt over a list of host (CPU, float32) matrices of one shape with
    the copies overlapped (pinned tensors for overlap).  Returns the list of
    outputs (allocated pinned if not given).  Asynchronous on `stream`:
    synchronise it before reading the outputs."""
    import torch
    if not Xs:
        return []
    m, n = Xs[0].shape
    for X in Xs:
        if X.is_cuda or X.dtype != torch.float32 or X.dim() != 2 or tuple(X.shape) != (m, n) or X.stride(1) != 1:
            raise ValueError("Xs must be host float32 m x n tensors with unit column stride")
    if Ys is None:
        Ys = [torch.empty((m, n), dtype=torch.float32, pin_memory=True) for _ in Xs]
    for Y in Ys:
        if Y.is_cuda or Y.dtype != torch.float32 or tuple(Y.shape) != (m, n) or Y.stride(1) != 1:
            raise ValueError("Ys must be host float32 m x n tensors with unit column stride")
    if len(Ys) != len(Xs) or len({X.stride(0) for X in Xs}) != 1 or len({Y.stride(0) for Y in Ys}) != 1:
        raise ValueError("Xs and Ys must have the same length and one row stride each")
    xp = (_vp * len(Xs))(*[ctypes.c_void_p(X.data_ptr()) for X in Xs])
    yp = (_vp * len(Ys))(*[ctypes.c_void_p(Y.data_ptr()) for Y in Ys])
    s = _as_shrink(shrink)
    sp = None
    if sparsify is not None:
        sp = ctypes.byref(CpaSparsify(int(sparsify[0]), int(sparsify[1]), float(sparsify[2]),
                                              int(sparsify[3]) if len(sparsify) > 3 else 0))
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt_host(h.ptr, len(Xs), xp, m, n, Xs[0].stride(0), ctypes.byref(s), int(L),
                               float(lambda_max), p, sp, yp, Ys[0].stride(0), _stream_ptr(stream)), "cpa_svt_host")
    return Ys


def cpa_get_lambda(h: Handle, stream=None) -> float:
    out = ctypes.c_double()
    _check(load().cpa_get_lambda(h.ptr, ctypes.byref(out), _stream_ptr(stream)), "cpa_get_lambda")
    return out.value


def cpa_sync_status(h: Handle, stream=None) -> int:
    """Device-side status of the last cpa_svt on the handle (synchronises
    the stream); returns the status code instead of raising."""
    return int(load().cpa_sync_status(h.ptr, _stream_ptr(stream)))


def cpa_get_coeffs(h: Handle, L: int, stream=None) -> np.ndarray:
    out = np.zeros(int(L), dtype=np.float64)
    _check(load().cpa_get_coeffs(h.ptr, out.ctypes.data_as(_P(_d)), int(L), _stream_ptr(stream)),
           "cpa_get_coeffs")
    return out


def cpa_profile_enable(h: Handle, enable: bool = True):
    _check(load().cpa_profile_enable(h.ptr, 1 if enable else 0), "cpa_profile_enable")


def cpa_profile_read(h: Handle, reset: bool = True) -> dict:
    ms = (ctypes.c_double * len(STAGES))()
    n = (ctypes.c_int64 * len(STAGES))()
    _check(load().cpa_profile_read(h.ptr, ms, n, 1 if reset else 0), "cpa_profile_read")
    return {st: {"ms": ms[i], "launches": n[i]} for i, st in enumerate(STAGES)}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def kernel_gemm_bf16(A_hi, A_lo, B_hi, B_lo, nsplit, D, sym=False, s_acc=1.0, C=None, s_c=0.0, C2=None, s_c2=0.0,
                     diag=0.0, H=None, coef=None, k=0, Dhi=None, Dlo=None, stream=None):
    """One tensor-core product with the fused epilogue (diagnostic entry)."""
    M, K = A_hi.shape
    N = B_hi.shape[0]
    _check(load().cpa_kernel_gemm_bf16(M, N, K, _ptr(A_hi), _ptr(A_lo), A_hi.stride(0), _ptr(B_hi), _ptr(B_lo),
                                       B_hi.stride(0), int(nsplit), 1 if sym else 0, float(s_acc), _ptr(C),
                                       float(s_c), _ptr(C2), float(s_c2), float(diag), _ptr(H), _ptr(coef), int(k),
                                       _ptr(D), D.stride(0), _ptr(Dhi), _ptr(Dlo),
                                       Dhi.stride(0) if Dhi is not None else 0, _stream_ptr(stream)),
           "cpa_kernel_gemm_bf16")


def kernel_split_bf16(X, transpose, hi, lo, stream=None):
    rows, cols = X.shape
    _check(load().cpa_kernel_split_bf16(_ptr(X), rows, cols, X.stride(0), 1 if transpose else 0, _ptr(hi),
                                        _ptr(lo), hi.stride(0), _stream_ptr(stream)), "cpa_kernel_split_bf16")


def kernel_topk_eps(Phi, k, stream=None):
    """The k-th largest |Phi_ij| of a square device matrix (cpa_kernel_topk_eps)."""
    p = Phi.shape[0]
    out = ctypes.c_float(0.0)
    _check(load().cpa_kernel_topk_eps(_ptr(Phi), p, Phi.stride(0), int(k), ctypes.byref(out), _stream_ptr(stream)),
           "cpa_kernel_topk_eps")
    return float(out.value)


class BatchPlan:
    """cpa_batch: shapes, offsets and term counts of a packed batch."""

    def __init__(self, h: Handle, shapes, offsets=None, L=None, L0: int = 24):
        self._lib = load()
        shapes = [(int(a), int(b)) for a, b in shapes]
        self.count = len(shapes)
        if offsets is None:
            offsets, o = [], 0
            for a, b in shapes:
                offsets.append(o)
                o += a * b
        self.shapes, self.offsets = shapes, list(offsets)
        self.L, self.L0 = (list(L) if L is not None else None), int(L0)
        self.total = max(o + a * b for (a, b), o in zip(shapes, self.offsets))
        off = (ctypes.c_int64 * self.count)(*self.offsets)
        ms = (ctypes.c_int32 * self.count)(*[a for a, _ in shapes])
        ns = (ctypes.c_int32 * self.count)(*[b for _, b in shapes])
        Ls = (ctypes.c_int32 * self.count)(*L) if L is not None else None
        ptr = ctypes.c_void_p()
        _check(self._lib.cpa_batch_create(h.ptr, self.count, off, ms, ns, Ls, int(L0), ctypes.byref(ptr)),
               "cpa_batch_create")
        self.ptr = ptr

    def close(self):
        if self.ptr:
            self._lib.cpa_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, variant=BATCH_MMA_SYNC, ctas_per_sm=0, order=ORDER_SIZE):
        _check(self._lib.cpa_batch_set_config(self.ptr, int(variant), int(ctas_per_sm), int(order)),
               "cpa_batch_set_config")

    def config(self):
        v, c, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.cpa_batch_get_config(self.ptr, ctypes.byref(v), ctypes.byref(c), ctypes.byref(o)),
               "cpa_batch_get_config")
        return v.value, c.value, o.value

    def tune_key(self, prec) -> str:
        """Key of the tuning cache: precision and the histogram of (p, q, L)."""
        import hashlib
        hist = {}
        for (m, n), L in zip(self.shapes, self.L if self.L is not None else [self.L0] * self.count):
            k = (min(m, n), max(m, n), int(L))
            hist[k] = hist.get(k, 0) + 1
        txt = "%s|%s" % (prec, sorted(hist.items()))
        return hashlib.sha1(txt.encode()).hexdigest()[:16]

    def tune(self, h, X, shrink, prec="bf16x3", reps=3, Y=None, cache=None, stream=None):
        """Picks the launch configuration of this plan: from the JSON file
        `cache` when it holds this plan's key, else by timing every
        candidate (cpa_batch_tune) and recording the choice there.  Returns
        (config, candidate times in ms or None)."""
        import json
        import torch
        key = self.tune_key(prec)
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if key in table:
            self.set_config(*table[key]["config"])
            return tuple(table[key]["config"]), None
        if Y is None:
            Y = torch.empty_like(X)
        arr, k = _shrink_array(shrink)
        chosen = (ctypes.c_int * 3)()
        ms = (ctypes.c_double * 8)()
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        _check(self._lib.cpa_batch_tune(h.ptr, self.ptr, ctypes.c_void_p(X.data_ptr()), arr, k, p,
                                        ctypes.c_void_p(Y.data_ptr()), int(reps), chosen, ms, _stream_ptr(stream)),
               "cpa_batch_tune")
        cfg = (chosen[0], chosen[1], chosen[2])
        times = [ms[i] for i in range(8)]
        if cache:
            table[key] = {"config": list(cfg), "ms": times}
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return cfg, times

    def lambdas(self, stream=None) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.float64)
        _check(self._lib.cpa_batch_read_lambdas(self.ptr, out.ctypes.data_as(_P(_d)), _stream_ptr(stream)),
               "cpa_batch_read_lambdas")
        return out


def cpa_svt_batched_plan(h: Handle, plan: BatchPlan, X, shrink, lambdas=None, iters: int = 20, prec="bf16x3", Y=None,
                    stream=None):
    """Batched shrinkage of the packed matrices in X (flat float32 CUDA
    tensor); shrink: one spec or a list with one per matrix; lambdas: None
    (computed on the device) or a float64 CUDA tensor of plan.count bounds."""
    import torch
    if not (X.is_cuda and X.dtype == torch.float32 and X.is_contiguous() and X.numel() >= plan.total):
        raise ValueError("X must be a contiguous float32 CUDA tensor covering the plan")
    if Y is None:
        Y = torch.empty_like(X)
    arr, k = _shrink_array(shrink)
    lam = None
    if lambdas is not None:
        if not (lambdas.is_cuda and lambdas.dtype == torch.float64 and lambdas.numel() == plan.count):
            raise ValueError("lambdas must be a float64 CUDA tensor of plan.count values")
        lam = ctypes.c_void_p(lambdas.data_ptr())
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt_batched_plan(h.ptr, plan.ptr, ctypes.c_void_p(X.data_ptr()), arr, k, lam, int(iters),
                                       p, ctypes.c_void_p(Y.data_ptr()), _stream_ptr(stream)), "cpa_svt_batched_plan")
    return Y


class MLP:
    """The predictor network (cpa_mlp): forward, gradients and Adam steps
    run in the library's kernels."""

    def __init__(self, sizes=(12, 64, 64, 2), seed: int = 1):
        self._lib = load()
        self.sizes = tuple(int(x) for x in sizes)
        ptr = ctypes.c_void_p()
        _check(self._lib.cpa_mlp_create(ctypes.byref(ptr), *self.sizes, ctypes.c_uint64(seed)), "cpa_mlp_create")
        self.ptr = ptr
        self.count = int(self._lib.cpa_mlp_param_count(self.ptr))

    def close(self):
        if self.ptr:
            self._lib.cpa_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.float32)
        _check(self._lib.cpa_mlp_get_params(self.ptr, out.ctypes.data_as(_P(ctypes.c_float)), self.count),
               "cpa_mlp_get_params")
        return out

    def set_params(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32)
        _check(self._lib.cpa_mlp_set_params(self.ptr, arr.ctypes.data_as(_P(ctypes.c_float)), self.count),
               "cpa_mlp_set_params")

    def forward(self, X, Y=None, stream=None):
        import torch
        if Y is None:
            Y = torch.empty((X.shape[0], self.sizes[-1]), dtype=torch.float32, device=X.device)
        _check(self._lib.cpa_mlp_forward(self.ptr, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                         ctypes.c_void_p(Y.data_ptr()), _stream_ptr(stream)), "cpa_mlp_forward")
        return Y

    def gradients(self, X, T, stream=None):
        g = np.zeros(self.count, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._lib.cpa_mlp_gradients(self.ptr, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                           X.shape[0], g.ctypes.data_as(_P(ctypes.c_float)), self.count,
                                           ctypes.byref(loss), _stream_ptr(stream)), "cpa_mlp_gradients")
        return g, loss.value

    def train_step(self, X, T, lr, weight_decay=0.0, want_loss=False, stream=None):
        loss = ctypes.c_float()
        _check(self._lib.cpa_mlp_train_step(self.ptr, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                            X.shape[0], float(lr), float(weight_decay),
                                            ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)),
               "cpa_mlp_train_step")
        return loss.value if want_loss else None


N_FEATURES = 12


class ShrinkArray:
    """Shrink parameters marshalled once into a C array, for repeated batched
    calls on the same plan (building the array per call costs host time
    proportional to the batch)."""

    def __init__(self, specs):
        specs = specs if isinstance(specs, (list, tuple)) else [specs]
        self.arr = (CpaShrink * len(specs))(*[_as_shrink(x) for x in specs])
        self.count = len(specs)


def _shrink_array(shrink):
    if isinstance(shrink, ShrinkArray):
        return shrink.arr, shrink.count
    specs = shrink if isinstance(shrink, (list, tuple)) else [shrink]
    return (CpaShrink * len(specs))(*[_as_shrink(x) for x in specs]), len(specs)


def cpa_batch_features(h: Handle, plan: BatchPlan, X, shrink, stream=None):
    """Predictor features (count x 12, float32 CUDA) and theta_4 (float64)."""
    import torch
    F = torch.empty((plan.count, N_FEATURES), dtype=torch.float32, device=X.device)
    th = torch.empty(plan.count, dtype=torch.float64, device=X.device)
    arr, k = _shrink_array(shrink)
    _check(load().cpa_batch_features(h.ptr, plan.ptr, ctypes.c_void_p(X.data_ptr()), arr, k,
                                     ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(th.data_ptr()),
                                     _stream_ptr(stream)), "cpa_batch_features")
    return F, th


def cpa_svt_batched_learned(h: Handle, plan: BatchPlan, net: MLP, X, shrink, L_scale=1.0, L_min=4, L_max=96,
                            L_fallback=50, use_lambda=False, margin=0.01, prec="bf16x3", Y=None, stream=None):
    import torch
    if Y is None:
        Y = torch.empty_like(X)
    arr, k = _shrink_array(shrink)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt_batched_learned(h.ptr, plan.ptr, net.ptr, ctypes.c_void_p(X.data_ptr()), arr, k,
                                          float(L_scale), int(L_min), int(L_max), int(L_fallback),
                                          1 if use_lambda else 0, float(margin), p,
                                          ctypes.c_void_p(Y.data_ptr()), _stream_ptr(stream)),
           "cpa_svt_batched_learned")
    return Y


def cpa_batch_read_choices(plan: BatchPlan, stream=None):
    Ls = (ctypes.c_int * plan.count)()
    nfb = ctypes.c_int()
    _check(load().cpa_batch_read_choices(plan.ptr, Ls, ctypes.byref(nfb), _stream_ptr(stream)),
           "cpa_batch_read_choices")
    return np.array(Ls[:], dtype=np.int64), nfb.value


class Admm:
    """cpa_admm: background-modelling ADMM around the shrinkage for m x n
    problems (the appendix ADMM Applicable Forms, Background Modeling)."""

    def __init__(self, h: Handle, m: int, n: int):
        self._lib = load()
        ptr = ctypes.c_void_p()
        _check(self._lib.cpa_admm_create(h.ptr, int(m), int(n), ctypes.byref(ptr)), "cpa_admm_create")
        self.ptr, self.m, self.n = ptr, int(m), int(n)

    def close(self):
        if self.ptr:
            self._lib.cpa_admm_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rpca(self, D, tau_nuclear, tau_l1, L, iters, prec="fp32", tol=0.0, Lout=None, Sout=None, stream=None,
             sparsify=None, schedule=False):
        """Returns (L, S, errors); D a float32 CUDA tensor m x n (row stride
        D.stride(0)); errors[t] = E after iteration t.  sparsify: None or
        (transform, mode, eps_or_frac); schedule: the kept fraction follows
        E_t (mode must be SPARSE_TOPK)."""
        import torch
        if not (D.is_cuda and D.dtype == torch.float32 and D.dim() == 2 and D.stride(1) == 1 and
                tuple(D.shape) == (self.m, self.n)):
            raise ValueError("D must be a float32 CUDA m x n tensor with unit column stride")
        Lout = torch.empty((self.m, self.n), dtype=torch.float32, device=D.device) if Lout is None else Lout
        Sout = torch.empty((self.m, self.n), dtype=torch.float32, device=D.device) if Sout is None else Sout
        done = ctypes.c_int()
        errs = (_d * int(iters))()
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        _check(self._lib.cpa_admm_rpca(self.ptr, ctypes.c_void_p(D.data_ptr()), D.stride(0), float(tau_nuclear),
                                       float(tau_l1), int(L), p,
                                       ctypes.byref(CpaSparsify(*sparsify)) if sparsify else None,
                                       1 if schedule else 0, int(iters), float(tol),
                                       ctypes.c_void_p(Lout.data_ptr()), ctypes.c_void_p(Sout.data_ptr()),
                                       ctypes.byref(done), errs, _stream_ptr(stream)), "cpa_admm_rpca")
        return Lout, Sout, np.array(errs[:done.value])


class Completion:
    """cpa_completion: the matrix completion ADMM of Section V, Comparison with Existing Methods (the inpainting
    problem without its average term) around the shrinkage for m x n
    problems."""

    def __init__(self, h: Handle, m: int, n: int):
        self._lib = load()
        ptr = ctypes.c_void_p()
        _check(self._lib.cpa_completion_create(h.ptr, int(m), int(n), ctypes.byref(ptr)), "cpa_completion_create")
        self.ptr, self.m, self.n = ptr, int(m), int(n)

    def close(self):
        if self.ptr:
            self._lib.cpa_completion_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, I, mask, tau_nuclear, tau_l1, L, iters, prec="fp32", tol=0.0, Lout=None, Z1out=None,
            stream=None):
        """Returns (l, z1 or None, errors); I a float32 CUDA tensor m x n,
        mask a uint8 CUDA tensor m x n (nonzero = observed), both with unit
        column stride."""
        import torch
        for t, dt, nm in ((I, torch.float32, "I"), (mask, torch.uint8, "mask")):
            if not (t.is_cuda and t.dtype == dt and t.dim() == 2 and t.stride(1) == 1 and
                    tuple(t.shape) == (self.m, self.n)):
                raise ValueError("%s must be a CUDA m x n tensor of %s with unit column stride" % (nm, dt))
        Lout = torch.empty((self.m, self.n), dtype=torch.float32, device=I.device) if Lout is None else Lout
        done = ctypes.c_int()
        errs = (_d * int(iters))()
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        _check(self._lib.cpa_completion_run(self.ptr, ctypes.c_void_p(I.data_ptr()), I.stride(0),
                                            ctypes.c_void_p(mask.data_ptr()), mask.stride(0), float(tau_nuclear),
                                            float(tau_l1), int(L), p, int(iters), float(tol),
                                            ctypes.c_void_p(Lout.data_ptr()), Lout.stride(0),
                                            ctypes.c_void_p(Z1out.data_ptr()) if Z1out is not None else None,
                                            ctypes.byref(done), errs, _stream_ptr(stream)), "cpa_completion_run")
        return Lout, Z1out, np.array(errs[:done.value])


def cpa_set_option(h: Handle, option: int, value: int):
    _check(load().cpa_set_option(h.ptr, int(option), int(value)), "cpa_set_option")


def learn_rule(L_scale=1.0, margin=0.02, L_min=4, L_max=1024, L_fallback=50, use_lambda=True) -> CpaLearnRule:
    return CpaLearnRule(float(L_scale), float(margin), int(L_min), int(L_max), int(L_fallback),
                        1 if use_lambda else 0)


def cpa_svt_learned(h: Handle, net, X, shrink, rule: CpaLearnRule, prec="bf16x3", Y=None, stream=None):
    """cpa_svt with (Lambda_max, L) chosen on the device by the predictor
    network `net` (an MLP of widths 12, 64, 64, 2)."""
    import torch
    ptr, m, n, ld = _matrix(X, "X")
    if Y is None:
        Y = torch.empty((m, n), dtype=torch.float32, device=X.device)
    yptr, ym, yn, ldy = _matrix(Y, "Y")
    if (ym, yn) != (m, n):
        raise ValueError("Y shape mismatch")
    s = _as_shrink(shrink)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt_learned(h.ptr, net.ptr, ctypes.c_void_p(ptr), m, n, ld, ctypes.byref(s),
                                  ctypes.byref(rule), p, ctypes.c_void_p(yptr), ldy, _stream_ptr(stream)),
           "cpa_svt_learned")
    return Y


def cpa_get_order(h: Handle, stream=None):
    L, fb = ctypes.c_int(), ctypes.c_int()
    _check(load().cpa_get_order(h.ptr, ctypes.byref(L), ctypes.byref(fb), _stream_ptr(stream)), "cpa_get_order")
    return L.value, fb.value


def cpa_learn_features(h: Handle, X, shrink, F=None, theta=None, stream=None):
    """The 12 predictor features and theta_4 of one matrix (device tensors)."""
    import torch
    ptr, m, n, ld = _matrix(X, "X")
    if F is None:
        F = torch.empty(12, dtype=torch.float32, device=X.device)
    if theta is None:
        theta = torch.empty(1, dtype=torch.float64, device=X.device)
    s = _as_shrink(shrink)
    _check(load().cpa_learn_features(h.ptr, ctypes.c_void_p(ptr), m, n, ld, ctypes.byref(s),
                                     ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(theta.data_ptr()),
                                     _stream_ptr(stream)), "cpa_learn_features")
    return F, theta


class MemberList:
    """Marshalled member arrays of a pointer-form batch (device pointers,
    shapes, leading dimensions, shrinks), built once and reused."""

    def __init__(self, Xs, Ys, shrinks):
        if len(Xs) != len(Ys):
            raise ValueError("Xs and Ys must have the same length")
        self.count = len(Xs)
        xs, ys, ms, ns, lx, ly = [], [], [], [], [], []
        for X, Y in zip(Xs, Ys):
            xp, m, n, ld = _matrix(X, "X")
            yp, ym, yn, ldy = _matrix(Y, "Y")
            if (ym, yn) != (m, n):
                raise ValueError("Y shape mismatch")
            xs.append(xp)
            ys.append(yp)
            ms.append(m)
            ns.append(n)
            lx.append(ld)
            ly.append(ldy)
        c = self.count
        self.X = (_vp * c)(*[ctypes.c_void_p(v) for v in xs])
        self.Y = (_vp * c)(*[ctypes.c_void_p(v) for v in ys])
        self.m = (_i64 * c)(*ms)
        self.n = (_i64 * c)(*ns)
        self.ldx = (_i64 * c)(*lx)
        self.ldy = (_i64 * c)(*ly)
        self.shapes = list(zip(ms, ns))
        if isinstance(shrinks, (list, tuple)):
            if len(shrinks) != c:
                raise ValueError("one shrink per member, or a single one")
            self.shrink = (CpaShrink * c)(*[_as_shrink(x) for x in shrinks])
            self.s_count = c
        else:
            self.shrink = (CpaShrink * 1)(_as_shrink(shrinks))
            self.s_count = 1


def cpa_svt_batched(h: Handle, members: MemberList, L=None, L0: int = 24, lambdas=None, prec="bf16x3",
                    stream=None):
    """Plain CPA of every member (pointer form): patch-sized members in one
    persistent launch, the others through cpa_svt.  L: list of orders or
    None (L0); lambdas: list of host bounds or None (computed)."""
    c = members.count
    Ls = (ctypes.c_int * c)(*[int(v) for v in L]) if L is not None else None
    lam = (ctypes.c_double * c)(*[float(v) for v in lambdas]) if lambdas is not None else None
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_svt_batched(h.ptr, c, members.X, members.m, members.n, members.ldx, members.shrink,
                                  members.s_count, Ls, int(L0), lam, p, members.Y, members.ldy, _stream_ptr(stream)),
           "cpa_svt_batched")


def cpa_serve_learned(h: Handle, net, members: MemberList, rule: CpaLearnRule, prec="bf16x3", stream=None):
    """The learned choice of (Lambda_max, L) for every member (pointer form)."""
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().cpa_serve_learned(h.ptr, net.ptr, members.count, members.X, members.m, members.n, members.ldx,
                                    members.shrink, members.s_count, ctypes.byref(rule), p, members.Y,
                                    members.ldy, _stream_ptr(stream)), "cpa_serve_learned")


def cpa_serve_read(h: Handle, count: int, stream=None):
    """(L per member, Lambda_max per member, fallback count) of the last
    cpa_serve_learned call on the handle."""
    L = np.zeros(count, dtype=np.int32)
    lam = np.zeros(count, dtype=np.float64)
    fb = ctypes.c_int()
    _check(load().cpa_serve_read(h.ptr, int(count), L.ctypes.data_as(_P(ctypes.c_int)),
                                 lam.ctypes.data_as(_P(_d)), ctypes.byref(fb), _stream_ptr(stream)),
           "cpa_serve_read")
    return L, lam, fb.value
