"""The learned predictor's training labels (tests/golden/make_predictor_labels.py)
and its FP64 feature restatement (tests/predictor_data.py), pinned on the
CPU against the dense oracle and spectral facts."""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle as O
import predictor_data as D
from paper_1705_07112_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_predictor_labels",
                                               os.path.join(HERE, "golden", "make_predictor_labels.py"))
LAB = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(LAB)


def patch_members(seed_index, want, start=0):
    """Indices of the first `want` patch-shaped members (cheap for the dense
    oracle) of the serving mix of seed_index."""
    out, i = [], start
    while len(out) < want:
        if inputs.served_one(seed_index, i).family == 0:
            out.append(i)
        i += 1
    return out


def test_label_order_meets_the_target_on_the_dense_oracle():
    """Brute force: Algorithm 1 in FP64 at the labelled L* on the label's
    interval is within TOL of the exact shrinkage (the oracle's Jacobi SVD),
    and the next lower ladder order is not; unreachable labels miss TOL at
    the top of the ladder."""
    checked = 0
    for i in patch_members(301, 12):
        row = LAB.label_one((301, i))
        sm = inputs.served_one(301, i)
        X = sm.X.astype(np.float64)
        sp = sm.shrink
        s = O.Shrink(sp.kind, sp.tau, sp.c, sp.eps, sp.noise)
        lam = max(row[10], row[8] + row[9]) * (1.0 + LAB.MARGIN)
        ex = O.shrink_exact(X, s)
        den = np.linalg.norm(ex)
        L = int(row[13])
        assert row[11] >= -1e-12   # theta_4 <= sigma_max^2
        if L == LAB.L_NONE:
            top = LAB.LADDER[-1]
            assert np.linalg.norm(O.cpa(X, s, top, lam) - ex) / den > LAB.TOL
            continue
        assert abs(math.exp(row[12]) - L) <= 1e-9 * L
        assert np.linalg.norm(O.cpa(X, s, L, lam) - ex) / den <= LAB.TOL
        k = LAB.LADDER.index(L)
        if k > 0:
            assert np.linalg.norm(O.cpa(X, s, LAB.LADDER[k - 1], lam) - ex) / den > LAB.TOL
        checked += 1
    assert checked >= 4


def test_label_targets_from_their_definitions():
    """t0 = log(sigma_max^2 / theta_4) with theta_4 the Rayleigh quotient
    after four power products (brute force: explicit products with the Gram
    matrix) and sigma_max from LAPACK."""
    for i in patch_members(302, 3):
        row = LAB.label_one((302, i))
        X = inputs.served_one(302, i).X.astype(np.float64)
        G = X.T @ X if X.shape[0] >= X.shape[1] else X @ X.T
        v = O.start_vector(LAB.START_SEED, G.shape[0])
        v = v / np.linalg.norm(v)
        for _ in range(3):
            v = G @ v
            v = v / np.linalg.norm(v)
        th4 = float(v @ G @ v)
        r4 = float(np.linalg.norm(G @ v - th4 * v))
        assert abs(row[8] - th4) <= 1e-10 * th4 and abs(row[9] - r4) <= 1e-8 * th4
        smax2 = np.linalg.norm(X, 2) ** 2
        assert abs(row[11] - math.log(smax2 / th4)) <= 1e-10


@pytest.mark.parametrize("name", ["predictor_labels_train.npz", "predictor_labels_eval.npz"])
def test_stored_labels_reproduce(name):
    """A few rows of each committed label file recomputed from the oracle."""
    path = os.path.join(HERE, "golden", name)
    if not os.path.exists(path):
        pytest.skip("label file not generated")
    d = np.load(path)
    seed = int(d["seed_index"])
    for i in patch_members(seed, 3) + [int(j) for j in np.nonzero(d["family"] == 1)[0][:2]]:
        row = LAB.label_one((seed, i))
        for k, f in enumerate(LAB.FIELDS):
            assert np.isclose(d[f][i], row[k], rtol=1e-9, atol=1e-12), (name, i, f, d[f][i], row[k])


def test_reference_features_obey_spectral_bounds():
    mats, specs = D.generate(20, seed=33)
    for X, s in zip(mats, specs):
        f = D.reference_features(X, s)
        Xd = X.astype(np.float64)
        m, n = X.shape
        sv = np.linalg.svd(Xd, compute_uv=False)
        E = float(np.sum(sv ** 2))
        th4 = E / math.exp(f[2])
        lmin = th4 * math.exp(f[4])
        assert th4 <= sv[0] ** 2 * (1 + 1e-12)
        assert lmin >= sv[-1] ** 2 * (1 - 1e-9) and lmin <= th4 * (1 + 1e-12)
        assert abs(math.exp(f[6]) * th4 ** 2 - np.sum(sv ** 4)) <= 1e-9 * np.sum(sv ** 4)
        assert f[0] == math.log(min(m, n)) and f[1] == math.log(max(m, n) / min(m, n))
        assert f[8] >= -1e-12   # Rayleigh quotients grow along the power iteration
        assert (f[10], f[11]) == ((1.0, 0.0) if s.kind == O.HARD else (0.0, 1.0) if s.kind == O.WSOFT
                                  else (0.0, 0.0))
