"""The learned (Lambda_max, L) predictor: its features against an FP64
restatement, its decision rule against explicit choices, and its gain.

The network is trained on the GPU by the library's own kernels on oracle
labels (tests/predictor_data.py), served through cpa_svt_batched_learned,
and judged by the FP64 oracle's exact shrinkage.  The measure is the one the
predictor exists for: the fraction of matrices within 1e-2 relative
Frobenius error of the exact shrinkage at a given cost, against the method
without it (20-step power bound, one L for every matrix).
"""
import math

import numpy as np
import pytest

import predictor_data as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


def spec_dict(s):
    return dict(kind=s.kind, tau=s.tau, c=s.c, eps=s.eps, noise=s.noise)


def test_features_match_fp64_restatement(lib):
    import torch
    mats, specs = D.generate(300, seed=7)
    h = lib.Handle(0)
    plan = lib.BatchPlan(h, [m.shape for m in mats], L0=24)
    X = torch.from_numpy(D.pack(mats)).cuda()
    F, th = lib.cpa_batch_features(h, plan, X, [spec_dict(s) for s in specs])
    F = F.cpu().numpy().astype(np.float64)
    th = th.cpu().numpy()
    R = np.array([D.reference_features(m, s) for m, s in zip(mats, specs)])
    # shape and kind entries are exact
    assert np.array_equal(F[:, [10, 11]], R[:, [10, 11]])
    assert np.allclose(F[:, [0, 1]], R[:, [0, 1]], rtol=0, atol=1e-6)
    # log-ratios of FP32 Gram quantities: FP32 rounding of G and of the
    # power steps, relative 1e-5 at most for these well-scaled matrices
    for j in (2, 3, 6, 7, 8, 9):
        assert np.max(np.abs(F[:, j] - R[:, j])) <= 1e-3, (j, np.max(np.abs(F[:, j] - R[:, j])))
    # lower edge: lambda_min / theta_4 in absolute terms (the ratio can be
    # small, where its log amplifies rounding)
    assert np.max(np.abs(np.exp(F[:, 4]) - np.exp(R[:, 4]))) <= 1e-4
    assert np.max(np.abs(F[:, 5] - (F[:, 3] - F[:, 4]))) <= 1e-5
    th_ref = np.array([D.O.lambda_bound(m.astype(np.float64), 3, D.MARGIN,
                                        D.O.start_vector(D.START_SEED, min(m.shape)))["theta"] for m in mats])
    assert np.allclose(th, th_ref, rtol=1e-5, atol=0)
    plan.close()
    h.close()


@pytest.mark.parametrize("use_lambda", [False, True])
def test_decision_rule_matches_explicit_choices(lib, use_lambda):
    """The fused learned run takes exactly the L that the documented rule
    derives from cpa_mlp_forward on cpa_batch_features, and equals the plain
    batched run given those (Lambda_max, L)."""
    import torch
    mats, specs = D.generate(200, seed=8)
    sd = [spec_dict(s) for s in specs]
    shapes = [m.shape for m in mats]
    h = lib.Handle(0)
    net = lib.MLP((12, 64, 64, 2), seed=4)
    P = net.get_params()
    P[-2], P[-1] = 0.3, math.log(20.0)   # output biases: y0 ~ 0.3, y1 ~ log 20
    net.set_params(P)
    X = torch.from_numpy(D.pack(mats)).cuda()
    plan = lib.BatchPlan(h, shapes, L0=24)
    F, th = lib.cpa_batch_features(h, plan, X, sd)
    y = net.forward(F).cpu().numpy().astype(np.float64)
    th = th.cpu().numpy()
    L_scale, L_min, L_max, L_fb, margin = 1.3, 6, 40, 50, 0.01
    Lf = np.ceil(np.exp(y[:, 1]) * L_scale)
    L_exp = np.where(Lf > L_max, L_fb, np.maximum(Lf, L_min)).astype(int)
    Y1 = lib.cpa_svt_batched_learned(h, plan, net, X, sd, L_scale=L_scale, L_min=L_min, L_max=L_max,
                                     L_fallback=L_fb, use_lambda=use_lambda, margin=margin, prec="bf16x3")
    Ls, nfb = lib.cpa_batch_read_choices(plan)
    assert np.array_equal(Ls, L_exp)
    lam = None
    if use_lambda:
        # the predicted bound, never below (theta_4 + r_4)(1 + margin)
        r4 = np.array([D.O.lambda_bound(m.astype(np.float64), 3, 0.0,
                                        D.O.start_vector(D.START_SEED, min(m.shape)))["resid"] for m in mats])
        lp = th * np.exp(np.maximum(y[:, 0], 0.0)) * (1.0 + margin)
        fl = (th + r4) * 1.01
        lam = torch.from_numpy(np.maximum(lp, fl)).cuda()
    assert nfb == int(np.sum(Lf > L_max))
    ref_plan = lib.BatchPlan(h, shapes, L=[int(v) for v in L_exp])
    Y2 = lib.cpa_svt_batched_plan(h, ref_plan, X, sd, lambdas=lam, prec="bf16x3")
    torch.cuda.synchronize()
    if use_lambda:   # Lambda_max rounded on the device vs the host: ulps
        assert torch.allclose(Y1, Y2, rtol=1e-5, atol=1e-6)
    else:            # same arithmetic in another instantiation of the kernel
        assert torch.allclose(Y1, Y2, rtol=1e-6, atol=1e-7)
    # argument checks
    with pytest.raises(lib.CpaError):
        lib.cpa_svt_batched_learned(h, plan, net, X, sd, L_scale=0.0)
    with pytest.raises(lib.CpaError):
        lib.cpa_svt_batched_learned(h, plan, net, X, sd, L_max=1025)
    other = lib.MLP((12, 32, 64, 2), seed=1)
    with pytest.raises(lib.CpaError):
        lib.cpa_svt_batched_learned(h, plan, other, X, sd)
    other.close()
    for p_ in (plan, ref_plan):
        p_.close()
    net.close()
    h.close()


def _exact_job(a):
    seed_index, i = a
    import oracle as O2
    from paper_1705_07112_gb300 import inputs as I2
    sm = I2.served_one(seed_index, i)
    sp = sm.shrink
    s = O2.Shrink(sp.kind, sp.tau, sp.c, sp.eps, sp.noise)
    X = sm.X.astype(np.float64)
    lam = O2.lambda_bound(X, 20, 0.01, O2.start_vector(D.START_SEED, min(X.shape)))["lam"]
    errs = O2.spectral_errors(O2.singular_values(X), s, lam, LADDER)
    return O2.shrink_exact_lapack(X, s), errs


LADDER = [32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024]


def test_learned_bf16_beats_plain_fp32_at_1e3(lib):
    """The committed predictor on held-out matrices of the serving mix (the
    evaluation seed, not trained on): the learned (Lambda_max, L) with BF16
    split-precision products puts more matrices per second within 1e-3 of
    the exact shrinkage (the oracle's, through LAPACK's SVD) than plain FP32
    CPA at the smallest fixed order that reaches the same fraction within
    it (chosen by the oracle's FP64 error of each order)."""
    import multiprocessing as mp
    import os

    import torch
    from paper_1705_07112_gb300 import inputs, train_predictor
    seed, count = 200, 300
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        res = pool.map(_exact_job, [(seed, i) for i in range(count)], chunksize=1)
    exact = [r[0] for r in res]
    errs64 = np.array([r[1] for r in res])
    mix = inputs.served_mix(count, seed_index=seed)
    Xs = [torch.from_numpy(sm.X).cuda() for sm in mix]
    Yl = [torch.empty_like(X) for X in Xs]
    Yp = [torch.empty_like(X) for X in Xs]
    specs = [spec_dict(sm.shrink) for sm in mix]
    h = lib.Handle(0)
    net, pr = train_predictor.load_predictor()
    rule = lib.learn_rule(L_scale=pr["L_scale"], margin=pr["margin"], L_min=4, L_max=1024, L_fallback=50,
                          use_lambda=True)
    ml, mp_ = lib.MemberList(Xs, Yl, specs), lib.MemberList(Xs, Yp, specs)

    def frac(Ys):
        e = []
        for Y, ex, sm in zip(Ys, exact, mix):
            den = np.linalg.norm(ex)
            e.append(np.linalg.norm(Y.cpu().numpy().astype(np.float64) - ex) /
                     (den if den > 0 else np.linalg.norm(sm.X)))
        return float(np.mean(np.array(e) <= 1e-3))

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_l = timed(lambda: lib.cpa_serve_learned(h, net, ml, rule, prec="bf16x3"))
    f_l = frac(Yl)
    Ls, _, nfb = lib.cpa_serve_read(h, count)
    fr = (errs64 <= 1e-3).mean(axis=0)
    ok = [k for k in range(len(LADDER)) if fr[k] >= f_l]
    L_p = LADDER[ok[0] if ok else int(np.argmax(fr))]
    t_p = timed(lambda: lib.cpa_svt_batched(h, mp_, L0=L_p, prec="fp32"), reps=1)
    f_p = frac(Yp)
    good_l, good_p = f_l * count / t_l, f_p * count / t_p
    print("\nlearned BF16X3: %.1f%% within 1e-3, %.0f matrices/s, %.0f good/s, mean L %.0f, %d fallbacks"
          % (100 * f_l, count / t_l, good_l, float(np.mean(Ls)), nfb))
    print("plain FP32 L=%d: %.1f%% within 1e-3, %.0f matrices/s, %.0f good/s" % (L_p, 100 * f_p, count / t_p,
                                                                                good_p))
    assert f_l >= 0.4, f_l
    assert good_l > good_p, (good_l, good_p)
    net.close()
    h.close()


def test_training_code_path(lib):
    """The training script's pieces on a small subset of the committed
    labels: the features regenerate the labelled matrices (checksums), the
    network's loss falls under the library's AdamW steps, and folding the
    input standardisation into the first layer leaves the outputs as they
    were."""
    import os

    import torch
    from paper_1705_07112_gb300 import train_predictor as TP
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "predictor_labels_train.npz")
    lab = np.load(path)
    idx = np.arange(600)
    h = lib.Handle(0)
    F, th = TP.features_of(h, int(lab["seed_index"]), lab["i"][idx], checksums=lab["checksum"][idx])
    assert np.allclose(th, lab["theta4"][idx], rtol=1e-4)
    T = np.stack([lab["t0"][idx], lab["t1"][idx]], axis=1)
    net, mu, sd = TP.train(F, T, steps=600, batch=128)
    Fn = torch.from_numpy(((F - mu) / sd).astype(np.float32)).cuda()
    y0 = net.forward(Fn).cpu().numpy().astype(np.float64)
    rms = float(np.sqrt(np.mean((y0 - T) ** 2)))
    assert rms < float(np.std(T[:, 1])), (rms, float(np.std(T[:, 1])))
    net = TP.fold_standardisation(net, mu, sd)
    y1 = net.forward(torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    assert np.allclose(y1, y0, rtol=1e-4, atol=1e-4)
    net.close()
    h.close()
