"""Oracle labels of the learned (Lambda_max, L) predictor on the serving mix.

For matrix i of paper_1705_07112_gb300.inputs.served_one(seed_index, i) the
FP64 oracle gives:
  theta_4, r_4   the Rayleigh quotient and residual after four products of
                 the power iteration from the SplitMix64 start vector
                 (oracle.lambda_bound with 3 steps);
  sigma_max^2    from the singular values (oracle.singular_values);
  L*             the smallest order on the ladder from which every larger
                 ladder order gives a CPA within TOL of the exact shrinkage
                 (oracle.spectral_errors, the spectral error identity) on the
                 interval [0, lam_label], lam_label = max(sigma_max^2,
                 theta_4 + r_4) (1 + MARGIN): the bound the learned path serves
                 when its prediction is right or clamped; L_NONE when even the
                 largest order misses TOL.
Targets of the network: t0 = log(sigma_max^2 / theta_4), t1 = log L*.
TOL = 0.9e-3 leaves a tenth of the 1e-3 target to the arithmetic of the
BF16X3 path (measured near 1e-5).

    python tests/golden/make_predictor_labels.py --seed-index 100 --count 16000 \
        --out tests/golden/predictor_labels_train.npz
    python tests/golden/make_predictor_labels.py --seed-index 200 --count 2000 \
        --out tests/golden/predictor_labels_eval.npz

Only the oracle and the seeded input generator are used.
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LADDER = sorted({int(round(8 * 2 ** (i / 4.0))) for i in range(33)})   # 8 .. 2048, ratio 2^(1/4)
TOL = 0.9e-3
MARGIN = 0.02
L_NONE = 4096
START_SEED = 0x1705071120000000


def label_one(args):
    seed_index, i = args
    import oracle as O
    from paper_1705_07112_gb300 import inputs
    sm = inputs.served_one(seed_index, i)
    X = sm.X.astype(np.float64)
    m, n = X.shape
    p = min(m, n)
    sp = sm.shrink
    s = O.Shrink(sp.kind, sp.tau, sp.c, sp.eps, sp.noise)
    sv = O.singular_values(X)
    smax2 = float(sv[0]) ** 2
    b = O.lambda_bound(X, 3, 0.0, O.start_vector(START_SEED, p))
    th4, r4 = float(b["theta"]), float(b["resid"])
    lam = max(smax2, th4 + r4) * (1.0 + MARGIN)
    err = O.spectral_errors(sv, s, lam, LADDER)
    Lstar = L_NONE
    for k in range(len(LADDER) - 1, -1, -1):
        if err[k] > TOL:
            break
        Lstar = LADDER[k]
    return (i, m, n, sm.family, sp.kind, sp.tau, sp.c, sp.noise, th4, r4, smax2,
            math.log(smax2 / max(th4, 1e-300)), math.log(Lstar), Lstar, float(np.sum(sm.X, dtype=np.float64)))


FIELDS = ["i", "m", "n", "family", "kind", "tau", "c", "noise", "theta4", "r4", "smax2", "t0", "t1", "Lstar",
          "checksum"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed-index", type=int, required=True)
    ap.add_argument("--count", type=int, required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    t0 = time.time()
    jobs = [(a.seed_index, i) for i in range(a.count)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        rows = pool.map(label_one, jobs, chunksize=8)
    rows.sort()
    arr = {f: np.array([r[k] for r in rows]) for k, f in enumerate(FIELDS)}
    np.savez_compressed(a.out, seed_index=a.seed_index, ladder=np.array(LADDER), tol=TOL, margin=MARGIN,
                        L_none=L_NONE, **arr)
    print("%d labels in %.0f s -> %s" % (a.count, time.time() - t0, a.out))


if __name__ == "__main__":
    main()
