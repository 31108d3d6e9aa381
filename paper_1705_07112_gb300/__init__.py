"""GB300 (sm_103a) CPA singular value shrinkage (arXiv 1705.07112).

The compute path is libcpa.so (hand-written CUDA kernels behind the C ABI in
include/cpa.h); this package is its thin ctypes binding plus seeded
synthetic workloads.  Importing the package does not load the library;
the first call does, and raises if it is missing.
"""
from ._lib import (BF16, BF16X3, FP32, HARD, SOFT, TF32, WSOFT, Admm, BatchPlan, Completion, CpaError, Handle,  # noqa: F401
                   ShrinkArray,
                   cpa_coeffs, cpa_svt_batched, cpa_svt_batched_plan,
                   cpa_get_coeffs, cpa_get_lambda, cpa_lambda_bound, cpa_profile_enable, cpa_profile_read,
                   cpa_svt, cpa_svt_host, load, shrink_struct,
                   MemberList, cpa_serve_learned, cpa_serve_read, cpa_svt_learned, learn_rule)
