// Internal declarations shared by the translation units of libcpa.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/cpa.h"

namespace cpa {

// ---------------------------------------------------------------------------
// Shrinkage response h(x) of Eq. filter_response_ours, shared by the host
// coefficient routine and the device coefficient kernel of this library.
//   h(x) = (sqrt x - W(x)) / sqrt x  if sqrt x > thr(x), else 0,
//   HARD: W = 0, thr = tau;  SOFT: W = thr = tau;
//   WSOFT: W = thr = c / (sqrt(max(x - noise, 0)) + eps).
// ---------------------------------------------------------------------------
struct ShrinkParams {
    int kind;
    double tau, c, eps, noise;
};

__host__ __device__ inline double response(const ShrinkParams &s, double x) {
    double r = x > 0.0 ? sqrt(x) : 0.0;
    double W, thr;
    if (s.kind == CPA_HARD) {
        W = 0.0;
        thr = s.tau;
    } else if (s.kind == CPA_SOFT) {
        W = s.tau;
        thr = s.tau;
    } else {
        double s2 = x - s.noise;
        double sest = s2 > 0.0 ? sqrt(s2) : 0.0;
        W = s.c / (sest + s.eps);
        thr = W;
    }
    return r > thr ? (r - W) / r : 0.0;
}

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxTerms = 4096;
constexpr double kLambdaMargin = 0.01;
constexpr uint64_t kStartSeed = 0x1705071120000000ULL;
constexpr int kDefaultPowerIters = 20;

// ---------------------------------------------------------------------------
// Fused GEMM epilogue used by every dense product of the path:
//   v = s_acc * acc + s_c * C(i,j) + s_c2 * C2(i,j) + (i == j ? diag : 0)
//   D(i,j) = v;   if H: H(i,j) += coef[k] * v
// D and C may alias (the recurrence overwrites Psi_{k-2} with Psi_k).
// Optional BF16 hi/lo copies of v (hi = bf16(v), lo = bf16(v - hi)) are
// written for the tensor-core operand of the next product.
// symmetric_upper: the output is symmetric and only tiles meeting the upper
// triangle are computed.  SIMT kernel: every array is written in full.
// Tensor-core kernel: C, C2, H and D are read/written at the lower-triangle
// position (j,i), j >= i, so the FP32 arrays are valid in their lower
// triangle (D in full when sym_full_d), while the BF16 copies Dhi/Dlo are
// written in full (they are the next product's TMA operand).  General
// (non-symmetric) tensor-core outputs carry D only.
// ---------------------------------------------------------------------------
struct Epilogue {
    float *D = nullptr;
    int64_t ldd = 0;
    const float *C = nullptr;
    int64_t ldc = 0;
    const float *C2 = nullptr;
    int64_t ldc2 = 0;
    float s_acc = 1.f, s_c = 0.f, s_c2 = 0.f, diag = 0.f;
    float *H = nullptr;
    int64_t ldh = 0;
    const double *coef = nullptr;
    int k = 0;
    __nv_bfloat16 *Dhi = nullptr, *Dlo = nullptr;
    int64_t ldb = 0;
    int symmetric_upper = 0;
    int sym_full_d = 0;
    // diagonal term read on the device: diag + dcoef[dk] - (dk2 >= 0 ? dcoef[dk2] : 0)
    const double *dcoef = nullptr;
    int dk = 0, dk2 = -1;
    // device word that receives CPA_ERR_TIMEOUT when a bounded wait of the
    // tensor-core kernel gives up (null: a word of the current device)
    int *err = nullptr;
};

// Bounded waits of the cooperative launches (the power iteration's and the
// recurrence's grid barriers).  wait_cycles: clock cycles a block waits at a
// grid barrier before it records CPA_ERR_TIMEOUT (0: the default, about 2 s
// at 2 GHz).  stall != 0: the first grid barrier waits for one arrival more
// than the grid makes, so it can only end by that limit (for tests of the
// timeout path; the waits inside a CTA keep their own fixed limit).
struct WaitPolicy {
    long long wait_cycles = 0;
    int stall = 0;
};
constexpr long long kDefaultWaitCycles = 4000000000LL;
__host__ __device__ inline long long wait_limit(const WaitPolicy &w) {
    return w.wait_cycles > 0 ? w.wait_cycles : kDefaultWaitCycles;
}

// Raises the dynamic shared-memory limit of `func` to `bytes` on the current
// device.  The attribute belongs to the device, so it is set once per
// (device, kernel, size) under a lock, not once per process.
cudaError_t ensure_smem_limit(const void *func, int bytes);

// The diagonal term of an epilogue (host value plus the device coefficients).
__device__ __forceinline__ float epilogue_diag(const Epilogue &e) {
    float d = e.diag;
    if (e.dcoef) d += (float)(e.dcoef[e.dk] - (e.dk2 >= 0 ? e.dcoef[e.dk2] : 0.0));
    return d;
}

// SIMT FP32 GEMM: out(i,j) = epi(sum_k A(i,k) B(j,k)),  i < M, j < N, k < K.
// a_kmajor: A(i,k) = A[i*lda + k], else A[k*lda + i]; likewise B.
cudaError_t gemm_f32(int M, int N, int K, const float *A, int64_t lda, bool a_kmajor,
                     const float *B, int64_t ldb, bool b_kmajor, const Epilogue &e,
                     cudaStream_t st);

// Tensor-core GEMM (tcgen05 + TMA + TMEM).  Operands are BF16 K-major
// (row-major rows of K contiguous elements), given as hi and optional lo
// parts.  nsplit = 1: hi*hi.  nsplit = 3: hi*hi + hi*lo + lo*hi.
struct TcOperand {
    const __nv_bfloat16 *hi = nullptr, *lo = nullptr;
    int64_t ld = 0;    // elements
    int rows = 0;      // M (for A) or N (for B)
};
cudaError_t gemm_tc(int M, int N, int K, const TcOperand &A, const TcOperand &B, int nsplit,
                    const Epilogue &e, cudaStream_t st, int num_sms);

// All recurrence steps k_first <= k < k_end in one cooperative launch (grid
// barrier between steps).  A: the At operand.  e: the step-independent
// epilogue fields (s_acc, s_c, s_c2, H, ldh, coef, ldd, ldb, symmetric_upper).
// Step k writes Psi_k over Psi_{k-2} in z[k&1] and its BF16 copies in
// zhi/zlo[k&1]; it reads Psi_{k-1} from slot (k&1)^1.  bar: one device word.
// When the launch keeps the state in tensor memory (one tile per CTA) the
// FP32 ring is not written; with Clenshaw's sum the closing step is then
// applied inside the launch and *closed is set to 1.  kpad > p: the BF16
// operands (A and the ring's copies, row stride >= kpad) hold zeros in
// columns p .. kpad-1 and the products contract over kpad.
cudaError_t gemm_tc_recurrence(int p, const TcOperand &A, int nsplit, const Epilogue &e, int k_first, int k_end,
                               float *const z[2], __nv_bfloat16 *const zhi[2], __nv_bfloat16 *const zlo[2],
                               unsigned int *bar, cudaStream_t st, int num_sms, int clenshaw = 0, int L = 0,
                               int *closed = nullptr, int kpad = 0, const WaitPolicy &wp = WaitPolicy(),
                               const int *L_dev = nullptr, uint8_t *mask_buf = nullptr);
// mask_buf (optional, ceil(p/128) * ceil(kpad/64) bytes): the launch first
// records which 128-row x K-slice-group tiles of A are zero and skips their
// loads and products (the sparsity-based reduction's thresholded operand).

// Sparsity-based reduction helpers (sparsify.cu).
// scratch: 4p floats, needed by the DCT (its table of cosines).
cudaError_t make_transform(int type, int p, float *T, int64_t ld, cudaStream_t st, int num_sms, float *scratch);
// row_flags (optional, p ints): set to 1 for the rows that keep a nonzero
// entry (the support used by the compaction), 0 for the others.
cudaError_t threshold_entries(float *Phi, int p, int64_t ld, const float *eps_dev, float eps_host, cudaStream_t st,
                              int num_sms, double *removed2 = nullptr, int *row_flags = nullptr);
cudaError_t symmetrize_lower(float *S, int p, int64_t ld, cudaStream_t st, int num_sms);
cudaError_t topk_eps(const float *Phi, int p, int64_t ld, long long k, unsigned long long *counts, unsigned int *bar,
                     int *err, float *eps_out, cudaStream_t st, int num_sms);
constexpr int kTopkCounts = 4 * 256;   // counts scratch of topk_eps (unsigned long long)
// Compaction of a thresholded Phi_ to the block of its nonzero rows S (the
// identities in sparsify.cu's header): S (idx, ascending) and s = |S| on
// the device from the row flags the threshold wrote; the s x s block; rows
// S of T; the series' value c_out on the zero block; H += scale c on the
// diagonal; F += c T^T T for a transform type.
cudaError_t compact_support(const int *flags, int p, int *idx, int *s_dev, cudaStream_t st);
cudaError_t gather_block(const float *Phi, int64_t ld, const int *idx, int s, float *A, int64_t lda, cudaStream_t st,
                         int num_sms);
cudaError_t gather_rows(const float *T, int64_t ld, const int *idx, int s, int p, float *R, int64_t ldr,
                        cudaStream_t st, int num_sms);
cudaError_t zero_block_value(const double *c, int L, double sigma, double *c_out, cudaStream_t st);
cudaError_t diag_add(float *H, int s, int64_t ld, const double *c, double scale, cudaStream_t st);
cudaError_t add_transform_gram(float *F, int p, int64_t ld, int type, const double *c, cudaStream_t st);

// Elementwise conversion of a row-major FP32 matrix to BF16 hi/lo parts,
// optionally transposed (out is cols x rows then).
cudaError_t split_bf16(const float *X, int rows, int cols, int64_t ldx, bool transpose,
                       __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ldo, cudaStream_t st);

}  // namespace cpa

namespace cpa {

// Power-iteration bound (definition in cpa_lambda_bound's comment); out =
// {theta, r, trace, lambda, status}.  v0, v1: p floats; norm2: iters+2 doubles.
cudaError_t power_bound(const float *G, int64_t ldg, int p, int iters, float *v0, float *v1, double *norm2,
                        double *out, cudaStream_t st);
// The same bound with all iterations in one cooperative launch (grid
// barrier between iterations).  bar, err: device scratch words.  coef (L
// doubles, optional): the block that forms lambda also forms the
// coefficients on [0, lambda] for the response sp, as device_coeffs would.
cudaError_t power_bound_persistent(const float *G, int64_t ldg, int p, int iters, float *v0, float *v1,
                                   double *norm2, unsigned int *bar, int *err, double *out, cudaStream_t st,
                                   int num_sms, int L = 0, const ShrinkParams *sp = nullptr,
                                   double *coef = nullptr, const WaitPolicy &wp = WaitPolicy(),
                                   const int *start_idx = nullptr);
// start_idx (optional, p ints): the start vector's entry i is entry
// start_idx[i] of the standard one (the bound of a principal block,
// computed as the bound of the matrix it is the nonzero block of).
cudaError_t device_coeffs(const double *lam_dev, double lam_host, int L, const ShrinkParams &s, double *c,
                          cudaStream_t st);
// B_hat = (2/lambda) G - Id: Z1 = B_hat, H = c0/2 Id + c1 B_hat (FP32), and
// the operand of every recurrence product At = (2/lambda) G without the -Id
// (the recurrence's epilogue applies it exactly): in A as FP32 for the
// CUDA-core path, as BF16 hi/lo in Athi/Atlo for the tensor-core path, with
// Z1 as BF16 hi/lo; their columns p .. ldb-1, and those of the ring's other
// BF16 slot Z0hi/Z0lo when given, are set to zero.
// span > 0: the series' interval is [a, b] with b - a = span and
// sigma = (a + b) / (b - a): At = (2/span) G, B_hat = At - sigma Id (the
// guarded interval); span = 0: [0, lambda], sigma = 1.
cudaError_t shift_init(const float *G, int64_t ldg, int p, const double *lam, const double *c, int L, float *A,
                       float *Z1, float *H, int64_t ld, __nv_bfloat16 *Athi, __nv_bfloat16 *Atlo,
                       __nv_bfloat16 *Z1hi, __nv_bfloat16 *Z1lo, int64_t ldb, cudaStream_t st, int num_sms,
                       int clenshaw = 0, __nv_bfloat16 *Z0hi = nullptr, __nv_bfloat16 *Z0lo = nullptr,
                       double span = 0.0, double sigma = 1.0);
// Host FP64 coefficients of Eq. chebychev_coeff_shifted on [a, b] (the
// response is 0 for x <= 0).
void coeffs_interval(const ShrinkParams &s, int L, double a, double b, double *c);
// Clenshaw's closing step H = (b_0 - b_2) / 2 with b_0 in H and b_2 in B2
// (B2 null: b_2 = c[2] Id); lower triangle only when lower_only.
cudaError_t clenshaw_finish(float *H, const float *B2, int p, int64_t ld, const double *c, int lower_only,
                            cudaStream_t st, int num_sms);
// hi/lo split of a symmetric p x p matrix valid in its lower triangle, both
// triangles written.
cudaError_t split_sym_lower(const float *S, int p, int64_t lds, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ldo,
                            cudaStream_t st);
cudaError_t check_finite(const float *X, int64_t rows, int64_t cols, int64_t ldx, int *flag, cudaStream_t st,
                         int num_sms);

// Learned choice of (Lambda_max, L) for one matrix (learned.cu): features of
// the Gram matrix G (p x p, q the other side), the predictor network P
// (12 -> 64 -> 64 -> 2), the decision rule of cpa_svt_batched_learned and
// the coefficients of the chosen L on [0, Lambda_max] (c_k = 0 for
// L <= k < L_max).  out = {theta, r, trace, lambda, status}, L_out = {L,
// fallback}.  feat_only: write the 12 features and theta_4 and stop.
// v0, v1, u0, u1: round_up(p, 4) floats each; acc: learn_scratch_doubles
// (with tabg after it: 2 L_max + 8 doubles).
size_t learn_scratch_doubles(int L_max);
cudaError_t learn_bound(const float *G, int64_t ldg, int p, int q, const ShrinkParams &sp, const float *P,
                        double L_scale, double margin, int L_min, int L_max, int L_fallback, int use_lambda,
                        int feat_only, int iters, float *v0, float *v1, float *u0, float *u1, double *acc,
                        double *tabg, unsigned int *bar, int *err, double *out, int *L_out, float *feat,
                        double *theta_out, double *coef, cudaStream_t st, int num_sms, const WaitPolicy &wp);

// One member of a batched launch: element offset of X (and Y) in packed
// buffers, shape, order; or (pointer form, x != null) its own X and Y with
// row strides.
struct BatchDesc {
    int64_t off;   // element offset of X (and Y) in the packed buffers
    int m, n, L, pad;
    // per-matrix operands (pointer form): X and Y with their own row
    // strides; null x: the packed buffers at `off` with row stride n
    const float *x;
    float *y;
    int64_t ldx, ldy;
};

// Learned selection inside the batched launch: the network's parameters
// (layout W1[64][12], b1, W2[64][64], b2, W3[2][64], b3) and the rule that
// maps its outputs (y0, y1) to (Lambda_max, L).
struct LearnArgs {
    const float *P;
    double L_scale, margin;
    int L_min, L_max, L_fallback, use_lambda;
    int *L_out;       // L chosen per matrix
    int *nfallback;   // matrices that took the fallback
};


// Tensor-core batched launch (batched_tc.cu): members with min(m, n) <= 128
// and max(m, n) <= 4096, every product with the BF16 hi/lo split on tcgen05
// tiles, the recurrence state in tensor memory, one CTA per member at a
// time.  Arguments as the batched kernel's (learn: the learned choice).
constexpr int kTcBatchP = 128, kTcBatchQ = 4096;
cudaError_t launch_batched_tc(const BatchDesc *desc, const int *order, int count, const float *X, float *Y,
                              const ShrinkParams *shr, int shr_stride, const double *lam_in, double *lam_out,
                              int iters, int *status, const int *L_in, const LearnArgs &la, bool learn,
                              int num_sms, cudaStream_t st);

// Pointer form of the batched launch (batched.cu).  One member: device X
// (m x n, row stride ldx) and Y (row stride ldy), order L, its shrinkage.
// Members must satisfy min(m, n) <= 64, max(m, n) <= 128, L <=
// batched_max_terms().  lambda_host: NULL (bounds computed on the device)
// or count values.  net != NULL: the learned choice with `rule` (orders
// clamped to batched_max_terms()).
struct PtrItem {
    const float *x;
    float *y;
    int64_t ldx, ldy;
    int m, n, L;
    ShrinkParams shrink;
};
struct PtrPlan;
PtrPlan *ptr_plan_create(int device, int num_sms);
void ptr_plan_destroy(PtrPlan *pp);
cpa_status ptr_plan_run(PtrPlan *pp, int count, const PtrItem *items, const double *lambda_host, int prec,
                        const float *net, const cpa_learn_rule *rule, cudaStream_t st,
                        int variant = CPA_BATCH_MMA_SYNC);
const double *ptr_plan_lambdas(const PtrPlan *pp);
const int *ptr_plan_orders(const PtrPlan *pp);
const int *ptr_plan_fallbacks(const PtrPlan *pp);
const int *ptr_plan_status(const PtrPlan *pp);
int batched_max_terms();

// Device view of a predictor network: its parameter array, widths
// {in, h1, h2, out} and device (nullptr for a null handle).
const float *mlp_device_params(cpa_mlp m, int dims[4], int *device);

}  // namespace cpa
