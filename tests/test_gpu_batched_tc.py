"""The tensor-core batched kernel (one 128-row tcgen05 tile per member,
recurrence state in tensor memory) against the FP64 oracle, member by
member, across its shape range (p = min(m, n) <= 128; q = max(m, n) up to
2048, so the Gram matrix takes several 256-column chunks of X and the final
product several 256-column output chunks, with ragged last chunks), every
shrink kind, orders from 1 to 300, with the bound given and computed on the
device.  Tolerance as for every BF16 split-precision
result: 2e-3 relative Frobenius (measures ~1e-5)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
SEED = 0x1705071120000000
TOL = 2e-3

SHAPES = [(1, 1), (1, 7), (7, 1), (3, 200), (200, 3), (17, 100), (100, 17), (40, 64), (64, 64), (65, 63),
          (63, 65), (96, 250), (250, 96), (127, 255), (128, 128), (128, 256), (256, 128), (120, 121),
          (57, 513), (513, 57), (128, 1030), (1030, 128), (90, 2048)]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def members(seed):
    rng = np.random.default_rng(seed)
    mats = []
    for (m, n) in SHAPES:
        r = max(1, min(m, n) // 8)
        mats.append((rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) +
                     0.05 * rng.standard_normal((m, n))).astype(np.float32))
    return mats


def shrink_of(kind, lam):
    sig = np.sqrt(lam / 1.01)
    if kind == O.HARD:
        return O.Shrink(O.HARD, 0.3 * sig)
    if kind == O.SOFT:
        return O.Shrink(O.SOFT, 0.2 * sig)
    return O.Shrink(O.WSOFT, 0.0, c=0.05 * sig * sig, eps=1e-8, noise=0.01 * sig * sig)


@pytest.mark.parametrize("kind", [O.HARD, O.SOFT, O.WSOFT])
@pytest.mark.parametrize("given", [True, False])
def test_tensor_core_batch_matches_oracle(lib, kind, given):
    import torch
    mats = members(5 + kind)
    X64 = [m.astype(np.float64) for m in mats]
    # the bound a caller gives: 1.01 sigma_max^2 (from LAPACK), which covers
    # the spectrum, so a long series stays bounded (the 20-step power bound
    # can land below sigma_max^2 when the top two singular values are close,
    # and then T_k grows without bound, on both sides)
    lams = [1.01 * np.linalg.norm(X, 2) ** 2 for X in X64]
    specs = [shrink_of(kind, l) for l in lams]
    Xs = [torch.from_numpy(m).cuda() for m in mats]
    h = lib.Handle(0)
    for L in ((1, 2, 3, 24, 300) if given else (1, 2, 3, 24)):
        Ys = [torch.full_like(X, 7.0) for X in Xs]
        mem = lib.MemberList(Xs, Ys, [dict(kind=s.kind, tau=s.tau, c=s.c, eps=s.eps, noise=s.noise) for s in specs])
        lib.cpa_svt_batched(h, mem, L0=L, lambdas=lams if given else None,
                            prec="bf16x3")
        torch.cuda.synchronize()
        lam_dev = lams if given else None
        if not given:   # the device's own 20-step bound, checked against the oracle's definition
            lam_dev = [O.lambda_bound(X, 20, 0.01, O.start_vector(SEED, min(X.shape)))["lam"] for X in X64]
        for X, Y, s, lam, sh in zip(X64, Ys, specs, lam_dev, SHAPES):
            ref = O.cpa(X, s, L, lam)
            assert rel(Y.cpu().numpy().astype(np.float64), ref) <= TOL, (sh, kind, L, given)
    h.close()
