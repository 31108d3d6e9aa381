"""The learned choice of (Lambda_max, L) for one matrix of any size
(cpa_learn_features, cpa_svt_learned) and the serving router over a mixed
batch (cpa_serve_learned):

* the features against an FP64 restatement of their definition (the
  oracle's power steps);
* the device decision against the documented rule applied on the host to
  the network's output on those features (cpa_mlp_forward);
* the result against the oracle's Algorithm 1 at the chosen (Lambda_max, L)
  and against cpa_svt given the same choice;
* the router: patch-sized members take the batched kernel's learned mode,
  the others cpa_svt_learned, each with the same result as that entry point.
"""
import math

import numpy as np
import pytest

import oracle as O
import predictor_data as D
from paper_1705_07112_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16x3": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def spec_dict(s):
    return dict(kind=s.kind, tau=s.tau, c=s.c, eps=s.eps, noise=s.noise)


def oshrink(sp):
    return O.Shrink(sp.kind, sp.tau, sp.c, sp.eps, sp.noise)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


SHAPES = [(64, 50), (300, 170), (170, 300), (130, 129), (1000, 900), (5, 700)]


def members(shapes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for (m, n) in shapes:
        fam = 0 if (m, n) == (64, 50) else 1
        sm = inputs.served_matrix(rng, fam)
        if sm.X.shape != (m, n):   # same recipe at the listed shape
            r = max(1, min(5, min(m, n) // 4))
            s = 0.05
            edge = s * (math.sqrt(m) + math.sqrt(n))
            A = rng.standard_normal((m, r)); A /= np.linalg.norm(A, axis=0)
            B = rng.standard_normal((r, n)); B /= np.linalg.norm(B, axis=1)[:, None]
            g = np.sort(np.exp(rng.uniform(math.log(1.5), math.log(40.0), size=r)))[::-1]
            X = ((A * (g * edge)) @ B + s * rng.standard_normal((m, n))).astype(np.float32)
            sm = inputs.ServedMatrix(X, sm.shrink, fam, r, s)
        out.append(sm)
    return out


def test_single_features_match_fp64_restatement(lib):
    import torch
    h = lib.Handle(0)
    for sm in members(SHAPES, 3):
        X = torch.from_numpy(sm.X).cuda()
        F, th = lib.cpa_learn_features(h, X, spec_dict(sm.shrink))
        torch.cuda.synchronize()
        F = F.cpu().numpy().astype(np.float64)
        R = D.reference_features(sm.X, oshrink(sm.shrink))
        assert np.array_equal(F[[10, 11]], R[[10, 11]])
        assert np.allclose(F[[0, 1]], R[[0, 1]], rtol=0, atol=1e-6)
        for j in (2, 3, 6, 7, 8, 9):
            assert abs(F[j] - R[j]) <= 1e-3, (sm.X.shape, j, F[j], R[j])
        assert abs(math.exp(F[4]) - math.exp(R[4])) <= 1e-4, (sm.X.shape, F[4], R[4])
        X64 = sm.X.astype(np.float64)
        th_ref = O.lambda_bound(X64, 3, 0.01, O.start_vector(D.START_SEED, min(X64.shape)))["theta"]
        assert abs(float(th.cpu()[0]) - th_ref) <= 1e-5 * th_ref
    h.close()


@pytest.mark.parametrize("use_lambda", [True, False])
@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_single_decision_and_result(lib, use_lambda, prec):
    import torch
    h = lib.Handle(0)
    net = lib.MLP((12, 64, 64, 2), seed=9)
    P = net.get_params()
    P[-2], P[-1] = 0.25, math.log(40.0)   # y0 ~ 0.25, y1 ~ log 40
    net.set_params(P)
    rule = lib.learn_rule(L_scale=1.2, margin=0.02, L_min=5, L_max=300, L_fallback=50, use_lambda=use_lambda)
    for sm in members(SHAPES[1:], 5):
        X = torch.from_numpy(sm.X).cuda()
        spec = spec_dict(sm.shrink)
        F, th = lib.cpa_learn_features(h, X, spec)
        y = net.forward(F.reshape(1, 12)).cpu().numpy().astype(np.float64)[0]
        th = float(th.cpu()[0])
        Y = lib.cpa_svt_learned(h, net, X, spec, rule, prec=prec)
        L, fb = lib.cpa_get_order(h)
        lam = lib.cpa_get_lambda(h)
        Lr = math.exp(y[1]) * rule.L_scale
        Lf = math.ceil(Lr)
        L_exp = rule.L_fallback if Lf > rule.L_max else max(Lf, rule.L_min)
        # the features come from this call's own Gram product (FP32 CUDA
        # cores or BF16 split): the same order unless exp(y1) L_scale sits
        # within rounding of an integer
        if abs(Lr - round(Lr)) > 1e-3:
            assert L == L_exp, (sm.X.shape, L, L_exp)
        else:
            assert abs(L - L_exp) <= 1
        X64 = sm.X.astype(np.float64)
        p = min(X64.shape)
        if use_lambda:
            r4 = O.lambda_bound(X64, 3, 0.0, O.start_vector(D.START_SEED, p))["resid"]
            want = max(th * math.exp(max(y[0], 0.0)) * (1.0 + rule.margin), (th + r4) * 1.01)
            assert abs(lam - want) <= 1e-4 * want, (sm.X.shape, lam, want)
        else:
            want = O.lambda_bound(X64, 20, 0.01, O.start_vector(D.START_SEED, p))["lam"]
            assert abs(lam - want) <= 1e-4 * want, (sm.X.shape, lam, want)
        got = Y.cpu().numpy().astype(np.float64)
        ref = O.cpa(X64, oshrink(sm.shrink), L, lam)
        assert rel(got, ref) <= TOL[prec], (sm.X.shape, prec, rel(got, ref))
        Y2 = lib.cpa_svt(h, X, spec, L, lam, prec)
        torch.cuda.synchronize()
        assert rel(got, Y2.cpu().numpy().astype(np.float64)) <= 1e-5
    with pytest.raises(lib.CpaError):
        lib.cpa_svt_learned(h, net, X, spec, lib.learn_rule(L_max=5000), prec=prec)
    with pytest.raises(lib.CpaError):
        lib.cpa_svt_learned(h, net, X, spec, lib.learn_rule(L_fallback=2000, L_max=1000), prec=prec)
    net.close()
    h.close()


def test_router_members_match_their_paths(lib):
    """A mixed batch through cpa_serve_learned: each patch-sized member
    equals the batched learned plan's result, each larger member equals
    cpa_svt_learned's, and the read-back orders and bounds are theirs."""
    import torch
    h = lib.Handle(0)
    net = lib.MLP((12, 64, 64, 2), seed=4)
    P = net.get_params()
    P[-2], P[-1] = 0.2, math.log(60.0)
    net.set_params(P)
    rule = lib.learn_rule(L_scale=1.0, margin=0.02, L_min=5, L_max=400, L_fallback=50, use_lambda=True)
    mix = inputs.served_mix(40, seed_index=7)
    Xs = [torch.from_numpy(sm.X).cuda() for sm in mix]
    Ys = [torch.zeros_like(X) for X in Xs]
    specs = [spec_dict(sm.shrink) for sm in mix]
    mem = lib.MemberList(Xs, Ys, specs)
    lib.cpa_serve_learned(h, net, mem, rule, prec="bf16x3")
    Ls, lams, nfb = lib.cpa_serve_read(h, len(mix))
    # members the batched kernels take (tensor cores: p <= 128, q <= 4096);
    # the plan form holds the patch-sized ones among them
    batched = [i for i, sm in enumerate(mix) if min(sm.X.shape) <= 128 and max(sm.X.shape) <= 4096]
    small = [i for i in batched if min(mix[i].X.shape) <= 64 and max(mix[i].X.shape) <= 128]
    assert 0 < len(small) and len(batched) < len(mix)
    for i in batched:
        sp = mix[i].shrink
        ref = O.cpa(mix[i].X.astype(np.float64), O.Shrink(sp.kind, sp.tau, sp.c, sp.eps, sp.noise), int(Ls[i]),
                    float(lams[i]))
        assert rel(Ys[i].cpu().numpy().astype(np.float64), ref) <= TOL["bf16x3"], (mix[i].X.shape, Ls[i])
    plan = lib.BatchPlan(h, [mix[i].X.shape for i in small], L0=24)
    Xp = torch.from_numpy(np.concatenate([mix[i].X.ravel() for i in small])).cuda()
    Yp = lib.cpa_svt_batched_learned(h, plan, net, Xp, [specs[i] for i in small], L_scale=rule.L_scale,
                                     L_min=rule.L_min, L_max=rule.L_max, L_fallback=rule.L_fallback,
                                     use_lambda=True, margin=rule.margin, prec="bf16x3")
    Lp, _ = lib.cpa_batch_read_choices(plan)
    torch.cuda.synchronize()
    yp, o = Yp.cpu().numpy(), 0
    for k, i in enumerate(small):
        m, n = mix[i].X.shape
        assert np.array_equal(Ys[i].cpu().numpy(), yp[o:o + m * n].reshape(m, n))
        assert Ls[i] == Lp[k]
        o += m * n
    for i in range(len(mix)):
        if i in batched:
            continue
        Y1 = lib.cpa_svt_learned(h, net, Xs[i], specs[i], rule, prec="bf16x3")
        L1, _ = lib.cpa_get_order(h)
        # the bound's sums are added across blocks in any order: equal to
        # FP64 rounding, the results to FP32 rounding
        assert L1 == Ls[i] and abs(lib.cpa_get_lambda(h) - lams[i]) <= 1e-12 * lams[i]
        assert rel(Y1.cpu().numpy().astype(np.float64), Ys[i].cpu().numpy().astype(np.float64)) <= 1e-6
    plan.close()
    net.close()
    h.close()


def test_router_streams_match_one_stream(lib):
    """The larger members on several streams (CPA_OPT_STREAMS) give the
    orders and results of one stream, and every member's call reports no
    device-side failure."""
    import torch
    h = lib.Handle(0)
    net = lib.MLP((12, 64, 64, 2), seed=4)
    P = net.get_params()
    P[-2], P[-1] = 0.2, math.log(60.0)
    net.set_params(P)
    rule = lib.learn_rule(L_scale=1.0, margin=0.05, L_min=5, L_max=400, L_fallback=50, use_lambda=True)
    mix = inputs.served_mix(60, seed_index=9)
    Xs = [torch.from_numpy(sm.X).cuda() for sm in mix]
    specs = [spec_dict(sm.shrink) for sm in mix]
    outs = []
    for streams in (1, 6):
        lib.cpa_set_option(h, lib.OPT_STREAMS, streams)
        Ys = [torch.zeros_like(X) for X in Xs]
        lib.cpa_serve_learned(h, net, lib.MemberList(Xs, Ys, specs), rule, prec="bf16x3")
        Ls, lams, _ = lib.cpa_serve_read(h, len(mix))
        outs.append((Ls, lams, [Y.cpu().numpy().astype(np.float64) for Y in Ys]))
        # plain members too
        Yp = [torch.zeros_like(X) for X in Xs]
        lib.cpa_svt_batched(h, lib.MemberList(Xs, Yp, specs), L0=40, prec="bf16x3")
        outs[-1] = outs[-1] + ([Y.cpu().numpy().astype(np.float64) for Y in Yp],)
    (L1, l1, Y1, P1), (L6, l6, Y6, P6) = outs
    assert np.array_equal(L1, L6)
    assert np.allclose(l1, l6, rtol=1e-12)
    for a, b in zip(Y1, Y6):
        assert rel(a, b) <= 1e-6
    for a, b in zip(P1, P6):
        assert rel(a, b) <= 1e-6
    lib.cpa_set_option(h, lib.OPT_STREAMS, 1)
    with pytest.raises(lib.CpaError):
        lib.cpa_set_option(h, lib.OPT_STREAMS, 65)
    net.close()
    h.close()


def test_member_sm_budget_keeps_results(lib):
    """Members' launches sized for a few SMs (CPA_OPT_MEMBER_SMS) on several
    streams give the results of full-GPU launches on one stream: the tile
    widths and grids change, and with them only the order of the FP32 sums
    of the split products (interleaved below BN = 256, by product at 256).
    Given bounds and orders, so the comparison is of the recurrence and
    products alone; the bar is a tenth of the BF16X3 tolerance against the
    oracle (2e-3), ten times the split arithmetic's measured error."""
    import torch
    h = lib.Handle(0)
    mix = inputs.served_mix(48, seed_index=11)
    Xs = [torch.from_numpy(sm.X).cuda() for sm in mix]
    specs = [spec_dict(sm.shrink) for sm in mix]
    lams = [1.02 * float(np.linalg.norm(sm.X.astype(np.float64), 2)) ** 2 for sm in mix]
    outs = []
    for streams, sms in ((1, 0), (6, 10), (6, 3)):
        lib.cpa_set_option(h, lib.OPT_STREAMS, streams)
        lib.cpa_set_option(h, lib.OPT_MEMBER_SMS, sms)
        Ys = [torch.zeros_like(X) for X in Xs]
        lib.cpa_svt_batched(h, lib.MemberList(Xs, Ys, specs), L0=60, lambdas=lams, prec="bf16x3")
        torch.cuda.synchronize()
        outs.append([Y.cpu().numpy().astype(np.float64) for Y in Ys])
    lib.cpa_set_option(h, lib.OPT_STREAMS, 1)
    lib.cpa_set_option(h, lib.OPT_MEMBER_SMS, 0)
    for other in outs[1:]:
        for a, b, sm in zip(outs[0], other, mix):
            assert rel(b, a) <= 1e-4, (sm.X.shape, rel(b, a))
    h.close()
