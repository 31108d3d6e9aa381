"""The device background-modelling ADMM (cpa_admm_rpca) against the FP64
oracle ADMM (oracle/admm.py): the same iteration with Algorithm 1 in FP64
as the shrinkage step, on the RPCA recipe of the 1024 x 1024 frame scaled
down (rank-r Gaussian factors with unit columns plus 5 % +-U[5,10]
outliers, rho = mn / (4 |D|_1), eta = 1 / sqrt(max(m, n)), L = 30)."""
import numpy as np
import pytest

from oracle import admm as A
from paper_1705_07112_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))


# Tolerances relative to the outputs: the shrinkage removes most of the
# energy of its input l + u1 here (|z1| is a few percent of it), so a
# per-call error of ~4e-6 of the input (BF16X3) is ~1e-4 of z1, and fifteen
# coupled iterations carry it on: 5e-3; FP32 (~3e-7 of the input): 2e-4.
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-4), ("bf16x3", 5e-3)])
@pytest.mark.parametrize("shape", [(96, 80, 5), (72, 130, 4)])
def test_admm_matches_the_oracle_cpa_run(lib, prec, tol, shape):
    import torch
    m, n, r = shape
    w = inputs.rpca_frame(m=m, n=n, rank=r)
    D = w.X.astype(np.float64)
    mu, eta, iters = w.meta["mu"], w.meta["eta"], 15
    Lr, Sr, Er = A.rpca_admm(D, eta / mu, iters + 1, A.svt_cpa(1.0 / mu, 30))
    Lo, So, _ = A.rpca_admm(D, eta / mu, iters, A.svt_cpa(1.0 / mu, 30))
    h = lib.Handle(0)
    ad = lib.Admm(h, m, n)
    Lg, Sg, E = ad.rpca(torch.from_numpy(w.X).cuda(), 1.0 / mu, eta / mu, 30, iters, prec=prec)
    torch.cuda.synchronize()
    assert rel(Lg.cpu().numpy(), Lo) <= tol, rel(Lg.cpu().numpy(), Lo)
    assert rel(Sg.cpu().numpy(), So) <= tol, rel(Sg.cpu().numpy(), So)
    # errors[t] is E of the least-squares iterate after iteration t: the
    # oracle's E[t + 1]
    assert len(E) == iters
    assert np.allclose(E, Er[1:iters + 1], rtol=50 * tol, atol=0)
    ad.close()
    h.close()


def test_admm_stops_on_tolerance(lib):
    import torch
    w = inputs.rpca_frame(m=64, n=48, rank=3)
    h = lib.Handle(0)
    ad = lib.Admm(h, 64, 48)
    mu, eta = w.meta["mu"], w.meta["eta"]
    D = torch.from_numpy(w.X).cuda()
    _, _, E_all = ad.rpca(D, 1.0 / mu, eta / mu, 30, 40)
    tol = float(E_all[9]) * 1.0001   # reached first after iteration 9 when E decreases
    first = int(np.argmax(E_all < tol))
    _, _, E = ad.rpca(D, 1.0 / mu, eta / mu, 30, 40, tol=tol)
    assert len(E) == first + 1 and E[-1] < tol and np.all(E[:-1] >= tol)
    with pytest.raises(lib.CpaError):
        ad.rpca(D, -1.0, eta / mu, 30, 5)
    with pytest.raises(ValueError):
        ad.rpca(D.t(), 1.0 / mu, eta / mu, 30, 5)
    ad.close()
    h.close()


def test_admm_full_frame_precisions(lib):
    """The 1024 x 1024 frame, 100 iterations, FP32, BF16X3 and BF16
    shrinkage: BF16X3 stays within 1e-2 of FP32; every run stays finite and
    its E falls.  (The plain-BF16 deviation is reported: its ~1e-4 per-call
    error, relative to the input, compounds over the loop.)"""
    import torch
    w = inputs.rpca_frame()
    mu, eta = w.meta["mu"], w.meta["eta"]
    h = lib.Handle(0)
    ad = lib.Admm(h, 1024, 1024)
    D = torch.from_numpy(w.X).cuda()
    Dn = w.X.astype(np.float64)
    out = {}
    for prec in ("fp32", "bf16x3", "bf16"):
        Lg, Sg, E = ad.rpca(D, 1.0 / mu, eta / mu, 30, 100, prec=prec)
        torch.cuda.synchronize()
        Ln, Sn = Lg.cpu().numpy().astype(np.float64), Sg.cpu().numpy().astype(np.float64)
        out[prec] = (Ln, E)
        res = np.linalg.norm(Ln + Sn - Dn) / np.linalg.norm(Dn)
        print("\n%s: E after 100 iterations %.3e, |L+S-D|/|D| %.3e" % (prec, E[-1], res), end="")
        assert np.all(np.isfinite(E)) and np.all(np.isfinite(Ln)) and E[-1] < E[5]
    d3 = rel(out["bf16x3"][0], out["fp32"][0])
    d16 = rel(out["bf16"][0], out["fp32"][0])
    print("\nrelative deviation from FP32: bf16x3 %.3e, bf16 %.3e" % (d3, d16))
    assert d3 <= 1e-2
    ad.close()
    h.close()


def test_admm_with_the_sparsity_schedule_matches_the_oracle(lib):
    """The ADMM with the sparsity-based reduction (DCT over the frame index)
    and the threshold schedule of Section V, Effects of Thresholding Value on smooth frames (96 frames, so the
    three kept fractions keep 1, 2 and 5 entries of the 96 x 96 Phi) against
    the FP64 oracle ADMM with the same schedule, FP32 shrinkage."""
    import math
    import torch
    D, mu, eta = inputs.smooth_video()
    m, n = D.shape
    p = min(m, n)
    T = np.zeros((p, p))
    for k in range(p):
        s = math.sqrt((1.0 if k == 0 else 2.0) / p)
        T[k] = s * np.cos(np.pi * (2 * np.arange(p) + 1) * k / (2 * p))
    iters = 16   # E_t falls below E_l = 0.03 at the fifteenth iterate
    Lo, So, Eo = A.rpca_admm(D.astype(np.float64), eta / mu, iters + 1, A.svt_cpa_sparse(1.0 / mu, 30, T),
                             schedule=True)
    Ld, _, _ = A.rpca_admm(D.astype(np.float64), eta / mu, iters, A.svt_cpa(1.0 / mu, 30))
    Lo, So, _ = A.rpca_admm(D.astype(np.float64), eta / mu, iters, A.svt_cpa_sparse(1.0 / mu, 30, T), schedule=True)
    h = lib.Handle(0)
    ad = lib.Admm(h, m, n)
    Dd = torch.from_numpy(D).cuda()
    Lg, Sg, E = ad.rpca(Dd, 1.0 / mu, eta / mu, 30, iters, prec="fp32", sparsify=(lib.T_DCT, lib.SPARSE_TOPK, 0.0),
                        schedule=True)
    torch.cuda.synchronize()
    assert rel(Lg.cpu().numpy(), Lo) <= 1e-3, rel(Lg.cpu().numpy(), Lo)
    assert rel(Sg.cpu().numpy(), So) <= 1e-3, rel(Sg.cpu().numpy(), So)
    assert np.allclose(E, Eo[1:iters + 1], rtol=1e-2)
    # the schedule reached more than one branch, and the reduction changed the result
    fr = sorted({A.eps_fraction(e) for e in Eo[:iters]})
    print("\nkept fractions used:", fr, " E:", ["%.2e" % e for e in Eo[:iters]])
    assert len(fr) >= 2
    assert rel(Lo, Ld) > 1e-3
    with pytest.raises(lib.CpaError):
        ad.rpca(Dd, 1.0 / mu, eta / mu, 30, 3, sparsify=(lib.T_DCT, lib.SPARSE_ABS, 0.1), schedule=True)
    ad.close()
    h.close()
