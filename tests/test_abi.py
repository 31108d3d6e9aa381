"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/cpa.h declares, and its host-side
coefficient routine matches the FP64 oracle; argument errors are reported
as status codes without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1705_07112_gb300 import _lib as L
from paper_1705_07112_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cpa.h")).read()
    return sorted(set(re.findall(r"CPA_API\s+[\w\s\*]+?\b(cpa_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cpa_coeffs", "cpa_lambda_bound", "cpa_svt", "cpa_svt_batched"]:
        assert required in names
    assert sorted(L.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name




@pytest.mark.parametrize("kind,tau,c,noise", [(O.HARD, 1.5, 0, 0), (O.SOFT, 0.7, 0, 0), (O.WSOFT, 0, 0.3, 0.2)])
@pytest.mark.parametrize("alpha,lam", [(1, 3.0), (2, 3.0), (20, 11.5), (50, 4096.0)])
def test_host_coeffs_match_oracle(lib, kind, tau, c, noise, alpha, lam):
    got = L.cpa_coeffs(L.shrink_struct(kind, tau, c, 1e-8, noise), alpha, lam)
    want = O.coeffs(O.Shrink(kind, tau, c, 1e-8, noise), alpha, lam)
    assert np.allclose(got, want, rtol=0, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_host_coeffs_argument_errors(lib):
    s = L.shrink_struct(L.SOFT, 1.0)
    out = (ctypes.c_double * 8)()
    assert lib.cpa_coeffs(ctypes.byref(s), 0, 1.0, out) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_coeffs(ctypes.byref(s), 8, 0.0, out) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_coeffs(ctypes.byref(s), 8, float("nan"), out) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_coeffs(ctypes.byref(s), 5000, 1.0, out) == L.CPA_ERR_INVALID_ARG
    bad = L.shrink_struct(L.SOFT, -1.0)
    assert lib.cpa_coeffs(ctypes.byref(bad), 8, 1.0, out) == L.CPA_ERR_INVALID_ARG
    bad = L.shrink_struct(7, 1.0)
    assert lib.cpa_coeffs(ctypes.byref(bad), 8, 1.0, out) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_coeffs(None, 8, 1.0, out) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_status_string(L.CPA_ERR_TIMEOUT).decode() == "device-side wait timed out"


def test_null_handle_is_rejected(lib):
    s = L.shrink_struct(L.SOFT, 1.0)
    out = ctypes.c_double()
    assert lib.cpa_svt(None, None, 4, 4, 4, ctypes.byref(s), 5, 0.0, 0, None, None, 4, None) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_lambda_bound(None, None, 4, 4, 4, 5, ctypes.byref(out), None) == L.CPA_ERR_INVALID_ARG
    assert lib.cpa_get_lambda(None, ctypes.byref(out), None) == L.CPA_ERR_INVALID_ARG


def test_tuning_cache_key_is_a_histogram():
    """The tuning cache key depends on the multiset of (p, q, L) and the
    precision only (not on the members' order or orientation)."""
    from paper_1705_07112_gb300 import _lib

    class P:   # the key's inputs without a device plan
        tune_key = _lib.BatchPlan.tune_key

    a, b, c = P(), P(), P()
    a.shapes, a.L, a.L0, a.count = [(64, 40), (40, 64), (64, 80)], None, 24, 3
    b.shapes, b.L, b.L0, b.count = [(64, 80), (64, 40), (64, 40)], None, 24, 3
    c.shapes, c.L, c.L0, c.count = [(64, 80), (64, 40), (64, 40)], [24, 24, 25], 24, 3
    assert a.tune_key("bf16x3") == b.tune_key("bf16x3")
    assert a.tune_key("bf16x3") != a.tune_key("fp32")
    assert c.tune_key("bf16x3") != b.tune_key("bf16x3")
