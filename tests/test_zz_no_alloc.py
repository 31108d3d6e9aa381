"""The allocation-free Lambda_max entry point (for callers that must not
allocate device memory: latency-critical loops, fixed memory budgets,
memory owned by another allocator) against the regular cpa_lambda_bound.

It is called through the C ABI twice in a row, on two different matrices,
so the second call runs on scratch that still holds the first call's data;
both results must match the regular entry point within the tolerance the
bound's parity tests use (1e-4 relative).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_bound_matches_regular_entry_twice():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib as L

    lib = L.load()
    h = L.Handle(0)
    rng = np.random.default_rng(2024)
    shapes = [(300, 170), (96, 512)]
    results = []
    for shape in shapes:
        X = (3.0 * rng.standard_normal((shape[0], 4)) @ rng.standard_normal((4, shape[1])) +
             0.1 * rng.standard_normal(shape)).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        out = ctypes.c_double()
        st = lib.cpa_lambda_bound_noalloc(ctypes.c_void_p(Xd.data_ptr()), shape[0], shape[1], Xd.stride(0), 20,
                                          ctypes.byref(out), stream)
        assert st == L.CPA_OK, L._status_string(st)
        ref = L.cpa_lambda_bound(h, Xd, 20)
        assert abs(out.value - ref) <= 1e-4 * ref, (shape, out.value, ref)
        results.append(out.value)
    assert results[0] != results[1]
    # sizes beyond the fixed scratch are refused, not truncated
    big = torch.zeros((600, 600), device="cuda")
    out = ctypes.c_double()
    st = lib.cpa_lambda_bound_noalloc(ctypes.c_void_p(big.data_ptr()), 600, 600, 600, 20, ctypes.byref(out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.CPA_ERR_INVALID_ARG
    h.close()


def test_noalloc_bound_at_the_size_limit_and_on_nonfinite_input():
    """min(m, n) = 512 exactly (the scratch array's largest Gram matrix)
    matches the regular entry point; one NaN entry gives CPA_ERR_NONFINITE
    through the status the bound's kernel leaves in the scratch array, and
    the call after it is again correct (the scratch is reused, not cleared
    by the caller)."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib as L

    lib = L.load()
    h = L.Handle(0)
    rng = np.random.default_rng(77)
    stream = lambda: ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)   # noqa: E731

    def noalloc(Xd, m, n):
        out = ctypes.c_double()
        st = lib.cpa_lambda_bound_noalloc(ctypes.c_void_p(Xd.data_ptr()), m, n, Xd.stride(0), 20,
                                          ctypes.byref(out), stream())
        return st, out.value

    for shape in [(700, 512), (512, 513)]:
        X = (2.0 * rng.standard_normal((shape[0], 3)) @ rng.standard_normal((3, shape[1])) +
             0.1 * rng.standard_normal(shape)).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        st, lam = noalloc(Xd, *shape)
        assert st == L.CPA_OK, L._status_string(st)
        ref = L.cpa_lambda_bound(h, Xd, 20)
        assert abs(lam - ref) <= 1e-4 * ref, (shape, lam, ref)
    Xn = torch.ones((64, 40), device="cuda")
    Xn[5, 7] = float("nan")
    st, _ = noalloc(Xn, 64, 40)
    assert st == L.CPA_ERR_NONFINITE
    X = rng.standard_normal((64, 40)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    st, lam = noalloc(Xd, 64, 40)
    assert st == L.CPA_OK and abs(lam - L.cpa_lambda_bound(h, Xd, 20)) <= 1e-4 * lam
    h.close()
