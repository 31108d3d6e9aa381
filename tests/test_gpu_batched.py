"""Parity of the batched path (cpa_svt_batched, one persistent launch) with
the FP64 oracle, matrix by matrix.

Tolerances as for the single-matrix path: fp32 1e-5; bf16 (hi/lo split in
every product) 2e-3 (measures ~1e-5).
"""
import numpy as np
import pytest

import oracle as O
from paper_1705_07112_gb300 import inputs

pytestmark = pytest.mark.gpu

SEED = 0x1705071120000000
TOL = {"fp32": 1e-5, "bf16": 2e-3, "bf16x3": 2e-3}


@pytest.fixture(scope="module")
def cpa():
    import __graft_entry__ as g
    g.build()
    import paper_1705_07112_gb300 as cpa
    return cpa


@pytest.fixture(scope="module")
def handle(cpa):
    h = cpa.Handle(0)
    yield h
    h.close()


def oracle_lambda(X64):
    return O.lambda_bound(X64, 20, 0.01, O.start_vector(SEED, min(X64.shape)))["lam"]


def pack(mats):
    import torch
    flat = np.concatenate([m.astype(np.float32).ravel() for m in mats])
    return torch.from_numpy(flat).cuda()


def unpack(Y, shapes):
    y = Y.cpu().numpy().astype(np.float64)
    out, o = [], 0
    for m, n in shapes:
        out.append(y[o:o + m * n].reshape(m, n))
        o += m * n
    return out


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


EDGE = [(1, 1), (1, 7), (7, 1), (64, 64), (64, 40), (40, 64), (17, 100), (100, 17), (128, 64), (64, 128),
        (3, 3), (63, 65), (65, 63), (16, 16), (33, 127)]


def edge_batch(seed=7):
    rng = np.random.default_rng(seed)
    mats = []
    for (m, n) in EDGE:
        r = max(1, min(m, n) // 6)
        mats.append(rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 0.05 * rng.standard_normal((m, n)))
    return mats


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("kind", [O.HARD, O.SOFT, O.WSOFT])
def test_batched_edge_shapes_given_lambda(cpa, handle, prec, kind):
    import torch
    mats = [m.astype(np.float32).astype(np.float64) for m in edge_batch()]
    shapes = [m.shape for m in mats]
    lams = np.array([oracle_lambda(m) for m in mats])
    specs = []
    for m, lam in zip(mats, lams):
        sig = np.sqrt(lam / 1.01)
        if kind == O.HARD:
            specs.append(O.Shrink(O.HARD, 0.3 * sig))
        elif kind == O.SOFT:
            specs.append(O.Shrink(O.SOFT, 0.2 * sig))
        else:
            specs.append(O.Shrink(O.WSOFT, 0.0, c=0.05 * sig * sig, eps=1e-8, noise=0.01 * sig * sig))
    Ls = [1, 2, 3, 24, 24, 24, 17, 17, 30, 30, 5, 24, 24, 9, 24]
    plan = cpa.BatchPlan(handle, shapes, L=Ls)
    Y = cpa.cpa_svt_batched_plan(handle, plan, pack(mats), [dict(kind=s.kind, tau=s.tau, c=s.c, eps=s.eps,
                                                            noise=s.noise) for s in specs],
                            lambdas=torch.tensor(lams, dtype=torch.float64, device="cuda"), prec=prec)
    torch.cuda.synchronize()
    for Xm, Ym, s, L, lam in zip(mats, unpack(Y, shapes), specs, Ls, lams):
        ref = O.cpa(Xm, s, L, lam)
        assert rel(Ym, ref) <= TOL[prec], (Xm.shape, L, rel(Ym, ref))
    assert np.array_equal(plan.lambdas(), lams)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_batched_computed_lambda(cpa, handle, prec):
    import torch
    mats = [m.astype(np.float32).astype(np.float64) for m in edge_batch(11)]
    shapes = [m.shape for m in mats]
    plan = cpa.BatchPlan(handle, shapes, L0=12)
    s = O.Shrink(O.SOFT, 0.5)
    Y = cpa.cpa_svt_batched_plan(handle, plan, pack(mats), dict(kind=O.SOFT, tau=0.5), prec=prec)
    torch.cuda.synchronize()
    lam_gpu = plan.lambdas()
    for i, (Xm, Ym) in enumerate(zip(mats, unpack(Y, shapes))):
        lam = oracle_lambda(Xm)
        assert abs(lam_gpu[i] - lam) <= 1e-4 * lam, (Xm.shape, lam_gpu[i], lam)
        assert rel(Ym, O.cpa(Xm, s, 12, lam)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp32"])
def test_patch_groups_full_batch_sampled(cpa, handle, prec):
    """The full 20,000-matrix patch-group batch in the benchmark's launch
    configuration (one persistent launch, device-computed bounds); a sample
    of matrices is checked against the oracle."""
    import torch
    mats, spec, L, sigma = inputs.patch_groups(20000)
    shapes = [m.shape for m in mats]
    specs = [dict(kind=spec.kind, tau=spec.tau, c=spec.c, eps=spec.eps,
                  noise=inputs.patch_group_noise(sh, sigma)) for sh in shapes]
    plan = cpa.BatchPlan(handle, shapes, L0=L)
    Y = cpa.cpa_svt_batched_plan(handle, plan, pack(mats), specs, prec=prec)
    torch.cuda.synchronize()
    lam_gpu = plan.lambdas()
    ys = unpack(Y, shapes)
    rng = np.random.default_rng(3)
    for i in list(rng.choice(len(mats), 60, replace=False)) + [0, len(mats) - 1]:
        Xm = mats[i].astype(np.float64)
        lam = oracle_lambda(Xm)
        assert abs(lam_gpu[i] - lam) <= 1e-4 * lam
        s = O.Shrink(specs[i]["kind"], 0.0, specs[i]["c"], specs[i]["eps"], specs[i]["noise"])
        assert rel(ys[i], O.cpa(Xm, s, L, lam)) <= TOL[prec], (i, Xm.shape)


def test_batch_plan_argument_errors(cpa, handle):
    with pytest.raises(cpa.CpaError):
        cpa.BatchPlan(handle, [(65, 65)])          # min(m, n) > 64
    with pytest.raises(cpa.CpaError):
        cpa.BatchPlan(handle, [(64, 129)])         # max(m, n) > 128
    with pytest.raises(cpa.CpaError):
        cpa.BatchPlan(handle, [(8, 8)], L0=0)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batched_long_series(cpa, handle, prec):
    """Orders above 128 (up to the kernel's limit of 1024): the coefficient
    sums run in the free Psi buffers; every member against the oracle."""
    import torch
    mats = [m.astype(np.float32).astype(np.float64) for m in edge_batch(seed=11)][:8]
    shapes = [m.shape for m in mats]
    Ls = [129, 200, 333, 512, 700, 1000, 1024, 300]
    specs = []
    for m in mats:
        sig = np.sqrt(oracle_lambda(m) / 1.01)
        specs.append(dict(kind=O.SOFT, tau=0.2 * sig))
    plan = cpa.BatchPlan(handle, shapes, L=Ls)
    Y = cpa.cpa_svt_batched_plan(handle, plan, pack(mats), specs, prec=prec)
    torch.cuda.synchronize()
    lam_gpu = plan.lambdas()
    for i, (Xm, y) in enumerate(zip(mats, unpack(Y, shapes))):
        s = O.Shrink(O.SOFT, specs[i]["tau"])
        ref = O.cpa(Xm, s, Ls[i], float(lam_gpu[i]))
        # FP32 arithmetic over up to 1024 terms: the recurrence's rounding
        # grows with the order, checked against the same 1e-5 bar
        assert rel(y, ref) <= TOL[prec], (i, Xm.shape, Ls[i], rel(y, ref))
    with pytest.raises(cpa.CpaError):
        cpa.BatchPlan(handle, [(8, 8)], L0=1025)
    plan.close()


def test_pointer_form_matches_plan_and_oracle(cpa, handle):
    """cpa_svt_batched (per-member device pointers, shapes, strides and
    orders): patch-sized members (one persistent launch) give exactly what
    the plan form gives; larger members (the single-matrix path) match
    the oracle; members are strided views of larger buffers."""
    import torch
    rng = np.random.default_rng(21)
    shapes = [(64, 40), (64, 80), (30, 100), (200, 150), (90, 300), (64, 64), (1, 9)]
    Ls = [24, 50, 10, 30, 17, 200, 5]
    mats, Xs, Ys = [], [], []
    for (m, n) in shapes:
        r = max(1, min(m, n) // 6)
        A = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 0.05 * rng.standard_normal((m, n)))
        A = A.astype(np.float32)
        mats.append(A.astype(np.float64))
        big = torch.zeros((m, n + 5), device="cuda")
        big[:, :n] = torch.from_numpy(A).cuda()
        Xs.append(big[:, :n])
        Ys.append(torch.full((m, n + 3), -3.0, device="cuda")[:, :n])
    lams = [oracle_lambda(A) for A in mats]
    specs = [dict(kind=O.SOFT, tau=0.2 * np.sqrt(l / 1.01)) for l in lams]
    for prec, tol in (("bf16x3", TOL["bf16x3"]), ("fp32", TOL["fp32"])):
        members = cpa.MemberList(Xs, Ys, specs)
        cpa.cpa_svt_batched(handle, members, L=Ls, lambdas=lams, prec=prec)
        torch.cuda.synchronize()
        small = [i for i, (m, n) in enumerate(shapes) if min(m, n) <= 64 and max(m, n) <= 128]
        plan = cpa.BatchPlan(handle, [shapes[i] for i in small], L=[Ls[i] for i in small])
        lam_t = torch.tensor([lams[i] for i in small], dtype=torch.float64, device="cuda")
        Yp = cpa.cpa_svt_batched_plan(handle, plan, pack([mats[i] for i in small]), [specs[i] for i in small],
                                      lambdas=lam_t, prec=prec)
        torch.cuda.synchronize()
        for k, y in zip(small, unpack(Yp, [shapes[i] for i in small])):
            assert np.array_equal(Ys[k].cpu().numpy().astype(np.float64), y), (prec, shapes[k])
        for i, A in enumerate(mats):
            ref = O.cpa(A, O.Shrink(O.SOFT, specs[i]["tau"]), Ls[i], lams[i])
            assert rel(Ys[i].cpu().numpy().astype(np.float64), ref) <= tol, (prec, shapes[i], rel(Ys[i].cpu().numpy(), ref))
        plan.close()


def test_launch_configurations_and_tuner(cpa, handle, tmp_path):
    """Every launch configuration of a plan (mma.sync kernel at 1 or 2 CTAs
    per SM, tcgen05 kernel; size-sorted or given work order) gives an
    oracle-accurate result; the tuner times them, keeps the fastest and
    records it in its JSON cache, which a second plan of the same shapes
    takes without timing."""
    import torch
    from paper_1705_07112_gb300 import _lib
    mats = [m.astype(np.float32).astype(np.float64) for m in edge_batch(seed=17)]
    shapes = [m.shape for m in mats]
    lams = np.array([oracle_lambda(m) for m in mats])
    specs = [dict(kind=O.SOFT, tau=0.2 * np.sqrt(l / 1.01)) for l in lams]
    X = pack(mats)
    plan = cpa.BatchPlan(handle, shapes, L0=30)
    refs = [O.cpa(m, O.Shrink(O.SOFT, s["tau"]), 30, l) for m, s, l in zip(mats, specs, lams)]
    lam_t = torch.from_numpy(lams).cuda()
    for cfg in [(0, 1, 0), (0, 2, 1), (1, 0, 0), (1, 0, 1)]:
        plan.set_config(*cfg)
        assert plan.config() == cfg
        Y = cpa.cpa_svt_batched_plan(handle, plan, X, specs, lambdas=lam_t, prec="bf16x3")
        torch.cuda.synchronize()
        for y, ref, sh in zip(unpack(Y, shapes), refs, shapes):
            assert rel(y, ref) <= TOL["bf16x3"], (cfg, sh)
    with pytest.raises(cpa.CpaError):
        plan.set_config(2, 0, 0)
    cache = str(tmp_path / "tune.json")
    cfg, ms = plan.tune(handle, X, specs, prec="bf16x3", reps=2, cache=cache)
    ran = [t for t in ms if t >= 0]
    assert len(ran) == 6 and plan.config() == cfg
    best = int(np.argmin([t if t >= 0 else np.inf for t in ms]))
    # candidate slots: variant x ctas_per_sm (1, 2) x order; the chosen one is the fastest
    assert cfg == (best // 4, 1 + (best // 2) % 2, best % 2)
    plan2 = cpa.BatchPlan(handle, shapes, L0=30)
    cfg2, ms2 = plan2.tune(handle, X, specs, prec="bf16x3", cache=cache)
    assert cfg2 == cfg and ms2 is None and plan2.config() == cfg
    plan.close()
    plan2.close()
