"""Failure detection on the device: a bounded wait that runs out.

The handle option CPA_OPT_STALL_TEST makes the first grid barrier of the
cooperative launches (the power iteration and the tensor-core recurrence)
wait for one arrival more than the grid makes: a flag that nothing sets.
With a short wait limit (CPA_OPT_WAIT_KCYCLES) the wait runs out, every
block records CPA_ERR_TIMEOUT and stops after its current step with its
copies drained and its tensor memory freed.  The tests check that the
status reaches the host through the C ABI and that the same handle then
computes a correct shrinkage: the context stays usable.  No kernel is
made to fault, trap or spin without a limit.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
SEED = 0x1705071120000000


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def _matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((m, 5)) @ rng.standard_normal((5, n)) +
            0.1 * rng.standard_normal((m, n))).astype(np.float32)


@pytest.mark.parametrize("shape", [(300, 256), (1024, 1024)])
def test_stalled_barrier_times_out_and_handle_recovers(lib, shape):
    import torch
    X = _matrix(*shape, seed=shape[0])
    X64 = X.astype(np.float64)
    p = min(shape)
    lam = O.lambda_bound(X64, 20, 0.01, O.start_vector(SEED, p))["lam"]
    s = O.Shrink(O.SOFT, 0.5 * 0.1 * (np.sqrt(shape[0]) + np.sqrt(shape[1])))
    spec = {"kind": s.kind, "tau": s.tau}
    Xd = torch.from_numpy(X).cuda()
    h = lib.Handle(0)
    try:
        lib.cpa_set_option(h, lib.OPT_WAIT_KCYCLES, 1000)   # about 0.5 ms per wait
        lib.cpa_set_option(h, lib.OPT_STALL_TEST, 1)
        # the recurrence's grid barrier (tensor-core path, bound given)
        lib.cpa_svt(h, Xd, spec, 20, lam, "bf16")
        assert lib.cpa_sync_status(h) == lib.CPA_ERR_TIMEOUT
        # the power iteration's grid barrier (bound computed on the device)
        lib.cpa_svt(h, Xd, spec, 20, 0.0, "fp32")
        assert lib.cpa_sync_status(h) == lib.CPA_ERR_TIMEOUT
        with pytest.raises(lib.CpaError) as ei:
            lib.cpa_lambda_bound(h, Xd, 20)
        assert ei.value.status == lib.CPA_ERR_TIMEOUT
        # back to normal operation on the same handle and context
        lib.cpa_set_option(h, lib.OPT_STALL_TEST, 0)
        lib.cpa_set_option(h, lib.OPT_WAIT_KCYCLES, 0)
        ref = O.cpa_vec(X64, s, 20, lam, X64[0] if shape[0] >= shape[1] else X64[:, 0])
        for prec, tol in (("bf16", 2e-3), ("fp32", 1e-5)):
            Y = lib.cpa_svt(h, Xd, spec, 20, lam, prec)
            assert lib.cpa_sync_status(h) == lib.CPA_OK
            got = Y.cpu().numpy().astype(np.float64)
            got = got[0] if shape[0] >= shape[1] else got[:, 0]
            scale = np.linalg.norm(Y.cpu().numpy()) / np.sqrt(max(shape))
            assert np.linalg.norm(got - ref) / max(np.linalg.norm(ref), scale) <= tol
        assert abs(lib.cpa_lambda_bound(h, Xd, 20) - lam) <= 1e-4 * lam
        with pytest.raises(lib.CpaError):
            lib.cpa_set_option(h, lib.OPT_STALL_TEST, 2)
        with pytest.raises(lib.CpaError):
            lib.cpa_set_option(h, lib.OPT_WAIT_KCYCLES, -1)
    finally:
        h.close()
