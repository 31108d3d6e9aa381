/*
 * cpa.h -- C ABI of the GB300 (sm_103a) library for CPA-based singular value
 * shrinkage (Onuki et al., "Fast Singular Value Shrinkage with Chebyshev
 * Polynomial Approximation Based on Signal Sparsity", arXiv 1705.07112).
 *
 * The library computes, for a real m x n matrix X,
 *
 *     G_hat(X) = X H_hat(X^T X)        (m >= n)
 *     G_hat(X) = H_hat(X X^T) X        (m <  n)
 *
 * with H_hat(G) = c_0/2 Id + sum_{k=1}^{L-1} c_k Psi_k(B_hat), B_hat =
 * (2/lambda_max) G - Id, the matrix Chebyshev polynomials Psi_k built by the
 * three-term recurrence Psi_k = 2 B_hat Psi_{k-1} - Psi_{k-2} (Section III-B,
 * Algorithm 1, Eqs. sing_shrink_from_eig_shrink, chebychev_series_matrix,
 * transform_lamB, cheby_matrix_eigen_saiki3, recurrence_our_method) and c_k
 * the shifted Chebyshev coefficients of h(x) = g(sqrt x)/sqrt x (Eq.
 * chebychev_coeff_shifted).  It approximates the exact shrinkage
 * G(X) = U diag(g(sigma_i)) V^T (Eq. sing_shrink_exact) without an SVD.
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major FP32 with a leading dimension in elements
 *     (ld >= number of columns).  Pointers named d* are DEVICE pointers
 *     owned by the caller; the library never frees them.
 *   - "L" is the number of Chebyshev terms (the paper's alpha): terms
 *     k = 0..L-1, polynomial degree L-1, L-2 recurrence products.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) unless they return a host value.
 *   - Every call returns a cpa_status and never throws or aborts.  On an
 *     argument error nothing is launched and no output is written.
 *   - A handle owns its device workspace; one handle must not be used from
 *     two host threads at once.  Different handles are independent.
 */
#ifndef CPA_H
#define CPA_H

#include <stdint.h>

#if defined(__GNUC__)
#define CPA_API __attribute__((visibility("default")))
#else
#define CPA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPA_OK = 0,
    CPA_ERR_INVALID_ARG = 1,   /* bad size, pointer, L, lambda or option        */
    CPA_ERR_CUDA = 2,          /* a CUDA runtime/driver call failed             */
    CPA_ERR_NO_MEMORY = 3,     /* workspace allocation failed                   */
    CPA_ERR_NONFINITE = 4,     /* NaN/Inf met in the input or the bound         */
    CPA_ERR_BOUND = 5,         /* lambda_max bound invalid (not > 0)            */
    CPA_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up            */
    CPA_ERR_UNSUPPORTED = 7    /* option not available on this device/build     */
} cpa_status;

/* Shrinkage kinds of the generic response h(x; W, tau) = (sqrt x - W)/sqrt x
 * when sqrt x > tau, else 0 (Section IV-A, Eq. filter_response_ours). */
typedef enum {
    CPA_HARD = 0,   /* W = 0,     threshold tau          g(s) = s [s > tau]     */
    CPA_SOFT = 1,   /* W = tau,   threshold tau          g(s) = max(s - tau, 0) */
    CPA_WSOFT = 2   /* W = w(x),  threshold w(x),  w(x) = c / (sqrt(max(x - noise, 0)) + eps) */
} cpa_kind;

/* Arithmetic of the dense products (Gram, recurrence, final product). */
typedef enum {
    CPA_FP32 = 0,    /* FP32 CUDA-core FMA throughout ("plain FP32 CPA")        */
    CPA_TF32 = 1,    /* tcgen05 kind::tf32 tensor cores, FP32 accumulate        */
    CPA_BF16 = 2,    /* tcgen05 kind::f16, FP32 accumulate: recurrence in BF16,
                        Gram and final product with the BF16 hi/lo split      */
    CPA_BF16X3 = 3   /* every product with the BF16 hi/lo split
                        (hi*hi + hi*lo + lo*hi), FP32 accumulate               */
} cpa_prec;

typedef struct {
    int kind;       /* cpa_kind                                                 */
    double tau;     /* HARD/SOFT threshold on sigma (>= 0)                      */
    double c;       /* WSOFT weight numerator (>= 0)                            */
    double eps;     /* WSOFT weight regulariser (> 0)                           */
    double noise;   /* WSOFT noise energy subtracted from sigma^2 (>= 0)        */
} cpa_shrink;

/* Optional sparsity-based reduction (Eqs. sing_shrink_exact_sparse and
 * threshold_components): Phi = T G T^T, entries with |Phi_ij| < eps set to 0,
 * result X T^T H_hat(Phi_) T (T^T H_hat T X for m < n).  Pass NULL for "off"
 * (T = Id, no threshold).  Transforms (p x p):
 *   HAAR1_LOWPASS: row i < floor(p/2) holds 1/sqrt2 at columns 2i, 2i+1; for
 *     odd p row floor(p/2) holds 1 at column p-1; the high band rows are 0.
 *   BLOCK_DCT8: block-diagonal orthonormal DCT-II, 8 x 8 blocks (the last
 *     block p mod 8 wide when that is not 0).
 *   DCT: orthonormal DCT-II, T[k][j] = s_k cos(pi (2j+1) k / 2p), s_0 =
 *     sqrt(1/p), s_k = sqrt(2/p).
 * Modes: ABS keeps |Phi_ij| >= eps_or_frac (>= 0); TOPK sets eps to the k-th
 * largest |Phi_ij|, k = ceil(frac p^2) in [1, p^2] (0 < frac <= 1), and keeps
 * the entries >= eps.  Phi, T and T^T H T are formed in FP32 on the device. */
typedef enum {
    CPA_T_IDENTITY = 0,
    CPA_T_HAAR1_LOWPASS = 1,   /* one-level Haar DWT, high band set to zero     */
    CPA_T_BLOCK_DCT8 = 2,      /* 8 x 8 block-diagonal orthonormal DCT-II       */
    CPA_T_DCT = 3              /* full orthonormal DCT-II                       */
} cpa_transform;

typedef enum {
    CPA_SPARSE_OFF = 0,        /* no entry threshold                            */
    CPA_SPARSE_ABS = 1,        /* keep |Phi_ij| >= eps_or_frac                  */
    CPA_SPARSE_TOPK = 2        /* eps = k-th largest |Phi_ij|, k = frac * p^2   */
} cpa_sparse_mode;

typedef struct {
    int transform;       /* cpa_transform                                        */
    int mode;            /* cpa_sparse_mode                                      */
    double eps_or_frac;  /* absolute threshold or fraction of entries kept       */
    int interval;        /* 0: the series on [0, Lambda_max] as Section III-B
                            writes it; 1: the guarded interval [a, b], a =
                            -|Phi - Phi_|_F, b = Lambda_max, which holds the
                            spectrum of the thresholded Phi_ (Weyl: its
                            eigenvalues are >= -|E|_2 >= -|E|_F), with
                            B_hat = (2 Phi_ - (a + b) Id) / (b - a) and the
                            coefficients of h on [a, b] (h = 0 for x <= 0);
                            the call then synchronises once to read a and b
                            and forms the coefficients on the host (FP64).
                            Ignored without an entry threshold.              */
} cpa_sparsify;

typedef struct cpa_ctx *cpa_handle;

/* Create a handle bound to CUDA device `device`.  Allocates nothing on the
 * device until the first call that needs workspace. */
CPA_API cpa_status cpa_create(cpa_handle *out, int device);

/* Free the handle and its workspace (synchronises the device first). */
CPA_API cpa_status cpa_destroy(cpa_handle h);

/* Static string for a status code. */
CPA_API const char *cpa_status_string(cpa_status s);

/* Text of the last CUDA failure seen by the calling thread ("" if none). */
CPA_API const char *cpa_last_error(void);

/* cpa_svt over a sequence of `count` host matrices of one shape: hX[i] (m x
 * n, row stride ldx) -> hY[i] (row stride ldy), other arguments as for
 * cpa_svt.  The handle stages two matrices on the device (4 m n floats,
 * allocated on first use) and overlaps the host-to-device copy of matrix
 * i + 1 and the device-to-host copy of matrix i - 1 with the shrinkage of
 * matrix i, on two copy streams of its own.  Asynchronous: `stream` waits for
 * the last copy, so a synchronisation of `stream` makes every hY valid.  The
 * copies overlap only for page-locked host memory (cudaMallocHost or
 * cudaHostRegister); pageable buffers work but serialise.  Host buffers must
 * not be touched until `stream` is synchronised.  Errors as cpa_svt, plus
 * INVALID_ARG for null or short buffers. */
CPA_API cpa_status cpa_svt_host(cpa_handle h, int count, const float *const *hX, int64_t m, int64_t n, int64_t ldx,
                                const cpa_shrink *s, int L, double lambda_max, int prec, const cpa_sparsify *sp,
                                float *const *hY, int64_t ldy, void *stream);

/* Shifted Chebyshev coefficients (Eq. chebychev_coeff_shifted), host FP64:
 *   c_k = (2/L) sum_{l=1}^{L} cos(k theta_l) h(lambda_max/2 (cos theta_l + 1)),
 *   theta_l = pi (l - 1/2)/L,  k = 0..L-1.
 * c_out: host array of L doubles.  Errors: INVALID_ARG if L < 1, L > 4096,
 * lambda_max not > 0, or the shrink parameters are out of range. */
CPA_API cpa_status cpa_coeffs(const cpa_shrink *s, int L, double lambda_max, double *c_out);

/* Upper estimate of Lambda_max, the largest eigenvalue of the Gram matrix G
 * of the smaller side of X (Algorithm 1's interval bound; the paper does not
 * say how it is computed).  Definition: `iters` power iterations
 * v <- G v / |G v| from the start vector v0_i = u_i - 1/2 (u_i output i of
 * SplitMix64 seeded with 0x1705071120000000, top 53 bits scaled to [0,1)),
 * then w = G v, theta = v.w, r = |w - theta v| and
 *     lambda = min((theta + r) * 1.01, trace G).
 * G is formed in FP32 on the device; theta, r and the trace are summed in
 * FP64.  Synchronises `stream` and writes the bound to *lambda_out (host).
 * Errors: INVALID_ARG (sizes, iters < 0), NONFINITE (NaN/Inf in X). */
CPA_API cpa_status cpa_lambda_bound(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx,
                            int iters, double *lambda_out, void *stream);

/* CPA singular value shrinkage of one matrix (Algorithm 1).
 *   dX: m x n input (device), dY: m x n output (device; must not overlap
 *   dX, INVALID_ARG otherwise), lambda_max: interval bound; <= 0 means "compute it on the
 *   device" with the definition of cpa_lambda_bound and iters = 20, in which
 *   case the coefficients are also formed on the device (FP64) and the whole
 *   call stays asynchronous.  prec: cpa_prec.  sp: NULL or sparsity option.
 * Errors: INVALID_ARG, UNSUPPORTED (prec not built for this device),
 * NO_MEMORY, CUDA.  Device-side failures of a computed bound (non-finite or
 * non-positive) are reported by the next cpa_get_lambda on the handle. */
CPA_API cpa_status cpa_svt(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx,
                   const cpa_shrink *s, int L, double lambda_max, int prec,
                   const cpa_sparsify *sp, float *dY, int64_t ldy, void *stream);

/* The Lambda_max used by the last cpa_svt on this handle (synchronises
 * `stream`).  Returns NONFINITE / BOUND if the device-computed bound was
 * not a positive finite number, TIMEOUT if a bounded device-side wait of
 * that call gave up (the output of that call is then unusable). */
CPA_API cpa_status cpa_get_lambda(cpa_handle h, double *lambda_out, void *stream);

/* Device-side status of the last cpa_svt on this handle: synchronises
 * `stream`, then returns CPA_OK, CPA_ERR_TIMEOUT (a bounded wait of one of
 * its kernels gave up: a grid barrier between steps, or a wait inside a
 * CTA; the kernels then stop, drain their copies in flight and release
 * their tensor memory, so the handle and the context stay usable),
 * CPA_ERR_NONFINITE or CPA_ERR_BOUND (the computed bound).  INVALID_ARG
 * before the first cpa_svt. */
CPA_API cpa_status cpa_sync_status(cpa_handle h, void *stream);

/* The L coefficients used by the last cpa_svt (synchronises `stream`). */
CPA_API cpa_status cpa_get_coeffs(cpa_handle h, double *c_out, int L, void *stream);

/* ---------------------------------------------------------------------------
 * Handle options (no counterpart in the paper).
 * CPA_OPT_SERIES: how cpa_svt sums the filter's series
 *   H_hat = c_0/2 Id + sum_{k=1}^{L-1} c_k T_k(B_hat):
 *   CPA_SERIES_FORWARD (default): Algorithm 1's forward recurrence
 *     Psi_k = 2 B_hat Psi_{k-1} - Psi_{k-2} with the running sum H += c_k Psi_k;
 *   CPA_SERIES_CLENSHAW: Clenshaw's recurrence b_k = c_k Id + 2 B_hat b_{k+1}
 *     - b_{k+2} (k = L-1 .. 0), H_hat = (b_0 - b_2) / 2: the same L-2
 *     products, no running sum (less memory traffic per step).  Its
 *     intermediates are larger than the filter they sum to, so with plain
 *     BF16 operands its error was measured at about 50 times the forward
 *     recurrence's (4e-3 to 6e-3 relative at p = 1000 .. 2048, L = 30),
 *     above the BF16 path's 2e-3 bar: cpa_svt with this series and
 *     CPA_BF16 returns CPA_ERR_UNSUPPORTED.  With CPA_BF16X3 or CPA_FP32
 *     its error is within 2x of the forward recurrence's.
 * Returns CPA_ERR_INVALID_ARG for an unknown option or value.
 * ------------------------------------------------------------------------- */
/* CPA_OPT_WAIT_KCYCLES: limit, in thousands of SM clock cycles, of the
 *   waits at the grid barriers between the steps of the cooperative launches
 *   (the power iteration and the tensor-core recurrence); 0 (the default)
 *   means 4,000,000 (about 2 s at 2 GHz).  When a wait runs out the kernel
 *   records CPA_ERR_TIMEOUT (read by cpa_sync_status, cpa_get_lambda or, for
 *   cpa_lambda_bound, its return value), stops, drains its copies in flight
 *   and frees its tensor memory: a failed call leaves the handle usable.
 * CPA_OPT_STALL_TEST: 1 makes the first grid barrier of those launches wait
 *   for one arrival more than the grid makes, so that it can end only by the
 *   limit above; for tests of the timeout path.  0 (the default) is normal
 *   operation. */
/* CPA_OPT_SPARSE_SKIP: 1 (the default) lets the tensor-core recurrence skip
 *   the tiles of the thresholded operand 2 Phi_ / Lambda_max that are zero
 *   (128 rows by 64 or 128 columns; the sparsity-based reduction with an
 *   entry threshold): their loads and products are not issued.  The skipped
 *   products are exact zeros, so the result is the same bit for bit; 0
 *   runs every tile (for comparisons). */
/* CPA_OPT_STREAMS: 1..64 (default 1): the pointer-form batches
 *   (cpa_svt_batched, cpa_serve_learned) run their larger members (those
 *   not taken by the batched kernel) round-robin on this many streams, each
 *   with a workspace of its own, forked from and joined back into the
 *   call's stream; matrices too small to fill the GPU then run side by
 *   side.  The results are those of one stream.  The device runs the work
 *   of at most CUDA_DEVICE_MAX_CONNECTIONS streams side by side (an
 *   environment variable read when the process first uses CUDA; 8 unless
 *   set, 32 at most): more streams than that share its work queues. */
/* CPA_OPT_MEMBER_SMS: >= 0 (default 0, all): the SMs each of those members'
 *   launches is sized for (tile widths and grids of its products, bound and
 *   recurrence), so that several large members run side by side instead of
 *   one after another; values above the device's SM count mean all.  The
 *   results do not depend on it beyond FP32 summation order. */
/* CPA_OPT_SPARSE_COMPACT: 1 (the default) lets a call with an entry
 *   threshold run the bound, shift and recurrence on the block Phi_[S, S]
 *   of the thresholded operand's nonzero rows S when |S| <= p / 2: every
 *   polynomial of Phi_ is that of the block on S and a constant c_out (the
 *   series at 0, or at the guarded interval's lower end mapped) elsewhere,
 *   so the filter is T_S^T (H_hat(Phi_[S,S]) - c_out Id) T_S + c_out T^T T
 *   with T_S the rows S of T, equal to the full recurrence's up to rounding;
 *   the call then synchronises once to read |S|.  The power iteration on
 *   the block starts from the entries S of the standard start vector, so
 *   the bound is that of Phi_.  0 runs the recurrence on the full p x p
 *   operand. */
enum { CPA_OPT_SERIES = 1, CPA_OPT_WAIT_KCYCLES = 2, CPA_OPT_STALL_TEST = 3, CPA_OPT_SPARSE_SKIP = 4,
       CPA_OPT_STREAMS = 5, CPA_OPT_MEMBER_SMS = 6, CPA_OPT_SPARSE_COMPACT = 7 };
enum { CPA_SERIES_FORWARD = 0, CPA_SERIES_CLENSHAW = 1 };
CPA_API cpa_status cpa_set_option(cpa_handle h, int option, int value);

/* ---------------------------------------------------------------------------
 * Diagnostics: per-stage device time and kernel-launch counts.
 * When enabled, every stage of cpa_svt is bracketed by CUDA events recorded
 * on the call's stream (each recurrence product separately), so the average
 * device time of one launch of a stage is ms[stage] / launches[stage].
 * Launch counts are kept whether or not timing is enabled.  Not for use while
 * the stream is being captured into a CUDA graph.
 * ------------------------------------------------------------------------- */
typedef enum {
    CPA_STAGE_PREP = 0,    /* FP32 -> BF16 hi/lo operand splits              */
    CPA_STAGE_GRAM = 1,    /* Gram product                                   */
    CPA_STAGE_BOUND = 2,   /* Lambda_max power iteration                     */
    CPA_STAGE_COEFF = 3,   /* device Chebyshev coefficients                  */
    CPA_STAGE_SHIFT = 4,   /* B_hat, Psi_1 and the initial sum               */
    CPA_STAGE_RECUR = 5,   /* recurrence products with fused accumulation    */
    CPA_STAGE_APPLY = 6,   /* final product                                  */
    CPA_STAGE_SPARSE = 7,  /* transform, entry threshold, T^T H T            */
    CPA_NSTAGES = 8
} cpa_stage;

CPA_API cpa_status cpa_profile_enable(cpa_handle h, int enable);

/* Synchronises the device; ms and launches: host arrays of CPA_NSTAGES
 * (either may be NULL), summed over the handle and the member streams of
 * its pointer-form batches (stage times of members that ran side by side
 * add up).  reset != 0 clears the accumulators afterwards. */
CPA_API cpa_status cpa_profile_read(cpa_handle h, double *ms, int64_t *launches, int reset);

/* ---------------------------------------------------------------------------
 * Kernel-level entry points used by the unit tests (no counterpart in the
 * paper): one tensor-core product with the fused epilogue, and one FP32 ->
 * BF16 hi/lo split.
 *   cpa_kernel_gemm_bf16: acc(i,j) = sum_k A(i,k) B(j,k) over the nsplit
 *   segments (1: hi*hi; 3: hi*hi + hi*lo + lo*hi), A: M x K and B: N x K
 *   row-major BF16 (ld multiple of 8, 16-byte aligned).
 *   sym = 0: D(i,j) = s_acc * acc + (i == j ? diag : 0), D: M x N FP32;
 *            C, C2, H, Dhi, Dlo must be NULL.
 *   sym = 1 (M == N, the output symmetric; only upper tiles are computed):
 *            v = s_acc acc + s_c C + s_c2 C2 + diag on the diagonal,
 *            D = v and H += coef[k] v in the LOWER triangle (row >= col;
 *            C, C2, H, D share ld = ldd), Dhi/Dlo = BF16 hi/lo of v in
 *            BOTH triangles (ld = ldh).  This is one recurrence step.
 *   cpa_kernel_split_bf16: hi = bf16(X), lo = bf16(X - hi), transposed
 *   (out is cols x rows) when transpose != 0.
 * ------------------------------------------------------------------------- */
CPA_API cpa_status cpa_kernel_gemm_bf16(int M, int N, int K, const void *A_hi, const void *A_lo, int64_t lda,
                                        const void *B_hi, const void *B_lo, int64_t ldb, int nsplit, int sym,
                                        float s_acc, const float *C, float s_c, const float *C2, float s_c2,
                                        float diag, float *H, const double *coef, int k, float *D, int64_t ldd,
                                        void *Dhi, void *Dlo, int64_t ldh, void *stream);
CPA_API cpa_status cpa_kernel_split_bf16(const float *X, int rows, int cols, int64_t ldx, int transpose, void *hi,
                                         void *lo, int64_t ldo, void *stream);
/* cpa_kernel_topk_eps: the entry threshold of CPA_SPARSE_TOPK alone: the
 * k-th largest |Phi_ij| (1 <= k <= p^2) of a p x p device matrix (ld >= p),
 * the 𝒦(|Phi|, k) of Eq. recommendation_epsilon, to *eps_host.  Allocates
 * and frees its scratch and synchronises `stream`. */
CPA_API cpa_status cpa_kernel_topk_eps(const float *Phi, int p, int64_t ld, long long k, float *eps_host,
                                       void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free Lambda_max bound.  The paper has no counterpart: this is a
 * deployment variant of cpa_lambda_bound for callers that cannot allocate
 * device memory (latency-critical loops that cannot pay for the device-wide
 * synchronisation of cudaMalloc/cudaFree, services held to a fixed device
 * memory budget, processes whose device memory belongs to another
 * allocator).  It takes no handle and allocates nothing: its scratch lives in
 * one fixed array of a little over 1 MB in device global memory that every
 * GPU loading the library holds until the process exits.
 *   Same definition and result as cpa_lambda_bound (same kernels), on the
 *   current device; dX as there; writes the bound to *lambda_out (host) and
 *   synchronises `stream`.
 *   Limits: min(m, n) <= 512, iters <= 1000; larger sizes return
 *   CPA_ERR_INVALID_ARG.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   The address is kept for the life of the process: after a reset of the
 *   device's primary context (cudaDeviceReset) it is stale, so do not use
 *   this entry point on a device that the process has reset.
 *   Every call shares the one array: calls whose work overlaps on the GPU
 *   (other host threads, other streams) race on it and must be serialised
 *   by the caller.
 * ------------------------------------------------------------------------- */
CPA_API cpa_status cpa_lambda_bound_noalloc(const float *dX, int64_t m, int64_t n, int64_t ldx, int iters,
                                            double *lambda_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned predictor network (no counterpart in the paper: it chooses
 * Lambda_max and L for Algorithm 1 from cheap features).  A fully connected
 * in -> h1 -> h2 -> out network, ReLU hidden layers, FP32, widths <= 128.
 * Parameters, one FP32 array: W1[h1][in], b1[h1], W2[h2][h1], b2[h2],
 * W3[out][h2], b3[out].  Loss of a batch of B samples:
 *   (1/2B) sum_b sum_o (y_bo - t_bo)^2.
 * Training updates with Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected, step t counted from 1 per network) and decoupled weight decay:
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   P <- P - lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + weight_decay P).
 * dX: device [B][in], dY / dT: device [B][out].
 * ------------------------------------------------------------------------- */
typedef struct cpa_mlp_ctx *cpa_mlp;

/* Creates the network on the current device; weights uniform with variance
 * 2/fan_in from SplitMix64(seed), biases 0. */
CPA_API cpa_status cpa_mlp_create(cpa_mlp *out, int in, int h1, int h2, int out_dim, uint64_t seed);
CPA_API cpa_status cpa_mlp_destroy(cpa_mlp m);
CPA_API int64_t cpa_mlp_param_count(cpa_mlp m);
CPA_API cpa_status cpa_mlp_set_params(cpa_mlp m, const float *host, int64_t count);
CPA_API cpa_status cpa_mlp_get_params(cpa_mlp m, float *host, int64_t count);
CPA_API cpa_status cpa_mlp_forward(cpa_mlp m, const float *dX, int batch, float *dY, void *stream);
/* Loss gradient with respect to every parameter (host copy) and the loss;
 * synchronises `stream`. */
CPA_API cpa_status cpa_mlp_gradients(cpa_mlp m, const float *dX, const float *dT, int batch, float *host_grad,
                                     int64_t count, float *host_loss, void *stream);
/* One Adam step on a batch (lr > 0, weight_decay >= 0); host_loss
 * (optional, synchronises) receives the batch loss before the step. */
CPA_API cpa_status cpa_mlp_train_step(cpa_mlp m, const float *dX, const float *dT, int batch, float lr,
                                      float weight_decay, float *host_loss, void *stream);

/* ---------------------------------------------------------------------------
 * Batched shrinkage of many small independent matrices (patch groups), one
 * persistent launch.  The matrices live packed in one device buffer: matrix
 * i starts at element offset off[i] and is row-major m[i] x n[i] with
 * leading dimension n[i]; the output uses the same offsets in dY.
 *
 * A plan uploads the descriptor table once (shapes, offsets, per-matrix L);
 * the same plan can be run many times on new data, and a run can be captured
 * in a CUDA graph.  Supported shapes: 1 <= min(m,n) <= 64, max(m,n) <= 128,
 * 1 <= L <= 1024 (patch groups; larger matrices go through cpa_svt).
 * ------------------------------------------------------------------------- */
typedef struct cpa_batch_ctx *cpa_batch;

/* L: host array of count term counts, or NULL to use L0 for every matrix. */
CPA_API cpa_status cpa_batch_create(cpa_handle h, int count, const int64_t *off, const int32_t *m,
                            const int32_t *n, const int32_t *L, int L0, cpa_batch *out);
CPA_API cpa_status cpa_batch_destroy(cpa_batch b);

/* Run the batched shrinkage.
 *   s: one shrink for all matrices (s_count = 1) or one per matrix
 *      (s_count = count), host array.
 *   lambda: NULL to compute each bound on the device (power iteration with
 *      `iters` steps, definition of cpa_lambda_bound), or a DEVICE array of
 *      count doubles.
 *   prec: CPA_FP32 (FP32 FMA on the CUDA cores) or CPA_BF16 / CPA_BF16X3
 *      (tcgen05 tensor cores, one 128-row tile per member with the
 *      recurrence state in tensor memory, the BF16 hi/lo split in every
 *      product: at these sizes the single-BF16 recurrence would cost
 *      accuracy and save nothing).
 * Asynchronous on `stream`.  The shrink parameters are uploaded on the first
 * run of a plan and whenever they change: such a run synchronises `stream`
 * first and cannot be captured in a CUDA graph; runs with unchanged
 * parameters only launch the kernel (capturable). */
CPA_API cpa_status cpa_svt_batched_plan(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s,
                           int s_count, const double *lambda, int iters, int prec, float *dY,
                           void *stream);

/* Launch configuration of a plan (no counterpart in the paper).
 *   variant: CPA_BATCH_MMA_SYNC (warp-level BF16 MMA, state in registers,
 *     up to 2 CTAs per SM) or CPA_BATCH_TCGEN05 (one 128-row tcgen05 tile
 *     per member, state in tensor memory, 1 CTA per SM); CPA_FP32 runs
 *     always take the FP32 CUDA-core form of the first.
 *   ctas_per_sm: CTAs per SM of the mma.sync kernel (1 or 2; 0: its
 *     occupancy limit).
 *   order: CPA_ORDER_SIZE (largest estimated work first, the default) or
 *     CPA_ORDER_GIVEN (the plan's own order).
 * Defaults: CPA_BATCH_MMA_SYNC, 0, CPA_ORDER_SIZE.
 * cpa_batch_tune times every configuration on the given data (one warm-up
 * and `reps` timed runs each, CUDA events on `stream`; synchronises),
 * keeps the fastest in the plan and returns it in chosen[3]; ms (optional,
 * 8 doubles) receives the mean time of each candidate, slot variant * 4 +
 * (ctas_per_sm - 1) * 2 + order, negative for candidates not run (the
 * tcgen05 variant runs at 1 CTA per SM, and not for CPA_FP32).  dY receives
 * the last run's output. */
enum { CPA_BATCH_MMA_SYNC = 0, CPA_BATCH_TCGEN05 = 1 };
enum { CPA_ORDER_SIZE = 0, CPA_ORDER_GIVEN = 1 };
CPA_API cpa_status cpa_batch_set_config(cpa_batch b, int variant, int ctas_per_sm, int order);
CPA_API cpa_status cpa_batch_get_config(cpa_batch b, int *variant, int *ctas_per_sm, int *order);
CPA_API cpa_status cpa_batch_tune(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                                  int prec, float *dY, int reps, int *chosen, double *ms, void *stream);

/* Per-matrix Lambda_max used by the last run of the plan (device array of
 * count doubles owned by the plan; valid until cpa_batch_destroy). */
CPA_API const double *cpa_batch_lambdas(cpa_batch b);

/* Copies those count values to host memory (synchronises `stream`); also
 * returns CPA_ERR_NONFINITE if a computed bound met a NaN/Inf. */
CPA_API cpa_status cpa_batch_read_lambdas(cpa_batch b, double *host_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned choice of (Lambda_max, L) for a batch (no counterpart in the
 * paper).  Features of matrix i (12 floats, dF[i][0..11]), with G its Gram
 * matrix, E = trace G = |X|_F^2, theta_t the Rayleigh quotient of the power
 * iterate after t-1 steps from the SplitMix64 start vector (t products with
 * G, so theta_t <= Lambda_max), r_4 = |G v - theta_4 v| for that unit
 * iterate, lambda_min the Rayleigh quotient after 4 steps
 * u <- (theta_4 I - G) u / |.| from the SplitMix64 vector of seed
 * (0x1705071120000000 xor 0x5EED), thr the threshold on sigma (weighted
 * soft: w at sigma^2 = theta_4), each of theta_4, lambda_min, thr^2 and
 * |G|_F^2 clamped below by 1e-30 E (1e-30 E^2):
 *   log p, log(q/p), log(E/theta_4), log(thr^2/theta_4),
 *   log(lambda_min/theta_4), log(thr^2/lambda_min), log(|G|_F^2/theta_4^2),
 *   log(E/(p thr^2)), log(theta_4/theta_2), log((theta_4 + r_4)/theta_4),
 *   [kind == HARD], [kind == WSOFT];   dTheta[i] = theta_4.
 * cpa_svt_batched_learned is one persistent launch that, per matrix,
 * computes the same features, runs the 12 -> 64 -> 64 -> 2 network `net`
 * (outputs y0 ~ log(sigma_max^2/theta_4), y1 ~ log L*; same FP32 results as
 * cpa_mlp_forward on the features) and shrinks with
 *   L = ceil(exp(y1) L_scale), at least L_min; L_fallback above L_max;
 *   Lambda_max = the 20-step power-iteration bound of cpa_lambda_bound, or,
 *     with use_lambda != 0, the prediction theta_4 exp(max(y0, 0))
 *     (1 + margin), never below the residual-corrected estimate
 *     (theta_4 + r_4)(1 + 0.01) (a bound below sigma_max^2 makes the
 *     series grow outside [-1, 1]).  With use_lambda only the features'
 *     four power products run, and a non-finite prediction falls back to
 *     the bound of those products, min((theta_5 + r_5)(1 + 0.01), trace G),
 *     with L_fallback.  The fallback count is of members that took
 *     L_fallback.
 * L_scale > 0, margin >= 0, 1 <= L_min <= L_max <= 1024, 1 <= L_fallback <=
 * 1024, else CPA_ERR_INVALID_ARG.  cpa_batch_read_choices returns the L used
 * per matrix and the number of fallbacks of the last learned run. */
CPA_API cpa_status cpa_batch_features(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                                      float *dF, double *dTheta, void *stream);
CPA_API cpa_status cpa_svt_batched_learned(cpa_handle h, cpa_batch b, cpa_mlp net, const float *dX,
                                           const cpa_shrink *s, int s_count, double L_scale, int L_min, int L_max,
                                           int L_fallback, int use_lambda, double margin, int prec, float *dY,
                                           void *stream);
CPA_API cpa_status cpa_batch_read_choices(cpa_batch b, int *host_L, int *host_fallbacks, void *stream);

/* The same learned choice for one matrix of any size (no counterpart in the
 * paper), inside the single-matrix shrinkage: cpa_svt with (Lambda_max, L)
 * chosen on the device.  The features are those of cpa_batch_features
 * computed from the Gram matrix of the call (FP32, power steps from the
 * same start vectors, |G|_F^2 and the trace summed in FP64); the network,
 * its output clamps and the decision rule are those of
 * cpa_svt_batched_learned with the rule's fields, L_fallback <= L_max <=
 * 4096.  Without use_lambda the 20-step bound of cpa_lambda_bound is used.
 * The coefficients of the chosen L are formed on the device in FP64 and the
 * recurrence reads L from device memory, so the call is asynchronous on
 * `stream` for CPA_BF16 / CPA_BF16X3 (CPA_FP32 synchronises once to read L).
 * The forward series only (CPA_ERR_UNSUPPORTED under CPA_SERIES_CLENSHAW).
 * cpa_get_order returns the L and the fallback flag (1 when the predicted
 * order exceeded L_max or the prediction was not finite) of the last
 * learned call; cpa_get_lambda its Lambda_max. */
typedef struct {
    double L_scale;   /* > 0: L = ceil(exp(y1) L_scale)                       */
    double margin;    /* >= 0: relative margin of the predicted bound          */
    int L_min, L_max, L_fallback;   /* 1 <= L_min <= L_max, 1 <= L_fallback <= L_max */
    int use_lambda;   /* serve the predicted bound (else the 20-step bound)    */
} cpa_learn_rule;
CPA_API cpa_status cpa_svt_learned(cpa_handle h, cpa_mlp net, const float *dX, int64_t m, int64_t n, int64_t ldx,
                                   const cpa_shrink *s, const cpa_learn_rule *rule, int prec, float *dY,
                                   int64_t ldy, void *stream);
CPA_API cpa_status cpa_get_order(cpa_handle h, int *L_out, int *fallback, void *stream);
/* ---------------------------------------------------------------------------
 * Batches given member by member: device pointers, shapes, leading
 * dimensions (elements, row-major) and orders per matrix, following the
 * problem statement of Algorithm 1 for each member.  Members with
 * min(m, n) <= 64, max(m, n) <= 128 and L <= 1024 run in one persistent
 * launch of the CUDA-core batched kernel (warp-level MMA); with CPA_BF16 /
 * CPA_BF16X3 the others with min(m, n) <= 128, max(m, n) <= 4096 and
 * L <= 1024 run in one persistent launch of the tcgen05 batched kernel; the
 * rest run through the single-matrix path (on CPA_OPT_STREAMS streams).  Asynchronous; the
 * descriptor table is uploaded on `stream` from pinned staging owned by the
 * handle (a later call waits until the previous upload has been read).
 * Members' X and Y must not overlap.  Errors: INVALID_ARG (any member),
 * UNSUPPORTED (precision), errors of cpa_svt pass through.
 *
 * cpa_svt_batched: plain CPA.  s: one shrink (s_count = 1) or one per
 *   member; L: host array of count orders or NULL (L0 for all); lambda:
 *   host array of count bounds (> 0) or NULL (each computed on the device
 *   with the definition of cpa_lambda_bound).
 * cpa_serve_learned: the learned choice of (Lambda_max, L) per member (no
 *   counterpart in the paper): the batched kernel's learned mode for the
 *   patch-sized members (orders clamped to 1024) and cpa_svt_learned for the
 *   others, the same network and rule for all.  cpa_serve_read returns, for
 *   the last learned call on the handle, each member's L and Lambda_max
 *   (host arrays of count, either may be NULL) and the number of members
 *   that took a fallback (synchronises `stream`).
 * ------------------------------------------------------------------------- */
CPA_API cpa_status cpa_svt_batched(cpa_handle h, int count, const float *const *dX, const int64_t *m,
                                   const int64_t *n, const int64_t *ldx, const cpa_shrink *s, int s_count,
                                   const int *L, int L0, const double *lambda, int prec, float *const *dY,
                                   const int64_t *ldy, void *stream);
CPA_API cpa_status cpa_serve_learned(cpa_handle h, cpa_mlp net, int count, const float *const *dX,
                                     const int64_t *m, const int64_t *n, const int64_t *ldx, const cpa_shrink *s,
                                     int s_count, const cpa_learn_rule *rule, int prec, float *const *dY,
                                     const int64_t *ldy, void *stream);
CPA_API cpa_status cpa_serve_read(cpa_handle h, int count, int *host_L, double *host_lambda, int *host_fallbacks,
                                  void *stream);

/* The 12 features and theta_4 of one matrix of any size (definition of
 * cpa_batch_features) into device memory dF[12], dTheta[1]; asynchronous. */
CPA_API cpa_status cpa_learn_features(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx,
                                      const cpa_shrink *s, float *dF, double *dTheta, void *stream);

/* ---------------------------------------------------------------------------
 * Background-modelling ADMM around the shrinkage (the appendix ADMM Applicable Forms, Background Modeling, Eq.
 * admm_algorithm_mod): min |l|_* + eta |s|_1 subject to l + s = d, with
 * rho the ADMM step.  Each iteration runs cpa_svt (soft threshold
 * tau_nuclear = 1/rho on the singular values, L terms, Lambda_max computed
 * on the device, precision `prec`) on l + u1, the entrywise soft threshold
 * tau_l1 = eta/rho on s + u2, the projection z3 = d, the dual update, and
 * the least-squares step l = (2a1 - a2 + a3)/3, s = (-a1 + 2a2 + a3)/3 with
 * a = z - u, all but the shrinkage in one fused elementwise kernel.  Start:
 * l = s = u = 1 (Section V, Background Modeling of Video).
 *
 * cpa_admm_create: solver for m x n problems on the handle's device; owns
 *   6 m n floats of state (m n <= 2^31).
 * cpa_admm_rpca: sp (optional) applies the sparsity-based reduction in every
 *   shrinkage; with schedule != 0 (sp->mode must be CPA_SPARSE_TOPK) the
 *   kept fraction follows the rule of Section V, Effects of Thresholding Value (Eq. recommendation_epsilon)
 *   on the current E_t: 0.5e-4 of p^2 while E_t > 0.03, 1.5e-4 while
 *   E_t > 6e-4, 0.5e-3 below (one host synchronisation per iteration).
 *   dD device m x n (row stride ldd >= n); dL, dS device m x n
 *   contiguous outputs, the last z1 (low-rank, exactly the shrinkage output)
 *   and z2 (sparse); they must not overlap each other or dD.  Runs
 *   max_iters iterations, or stops after iteration t when tol > 0 and
 *   E = |l_{t+2} - l_{t+1}|_F / |l_{t+2}|_F < tol (the check needs a host
 *   synchronisation per iteration; tol = 0 runs without one).
 *   *iters_done (optional) receives the iterations run; errors (optional,
 *   host, max_iters doubles) receives E after each iteration (synchronises).
 *   Errors: CPA_ERR_INVALID_ARG on bad arguments; errors of cpa_svt pass
 *   through. */
typedef struct cpa_admm_ctx *cpa_admm;
CPA_API cpa_status cpa_admm_create(cpa_handle h, int64_t m, int64_t n, cpa_admm *out);
CPA_API cpa_status cpa_admm_destroy(cpa_admm a);
CPA_API cpa_status cpa_admm_rpca(cpa_admm a, const float *dD, int64_t ldd, double tau_nuclear, double tau_l1, int L,
                                 int prec, const cpa_sparsify *sp, int schedule, int max_iters, double tol,
                                 float *dL, float *dS, int *iters_done, double *errors, void *stream);

/* ---------------------------------------------------------------------------
 * Matrix completion ADMM of Section V, Comparison with Existing Methods: the inpainting problem of
 * Section V, Texture Image Inpainting (Eq. texture_repaire4) without its average term, min |L|_* +
 * eta |Psi l|_1 subject to the observed entries and 0 <= L <= 1, in the
 * ADMM form of the appendix ADMM Applicable Forms, Texture Image Inpainting (Eq. admm_algorithm_inp without the z^(5) block):
 * z = K l, K = [Id; Psi; Omega; Id], Psi the orthonormal 2-D DCT (Psi l =
 * C_m L C_n^T, C_p[k][j] = s_k cos(pi (2j+1) k / (2p)), s_0 = sqrt(1/p),
 * s_k = sqrt(2/p)), Omega the observation mask.  Each iteration: the
 * least-squares step l = (a1 + Psi^T a2 + omega a3 + a4) / (3 + omega)
 * (a = z - u), z1 = cpa_svt(l + u1) (soft threshold tau_nuclear = 1/rho, L
 * terms, Lambda_max computed on the device, precision `prec`), z2 = the
 * entrywise soft threshold tau_l1 = eta/rho of Psi l + u2, z3 = the observed
 * values, z4 = l + u4 clipped to [0, 1], u += K l - z.  The four products
 * with C_m, C_n run in FP32 (prec = CPA_FP32) or on the tensor cores with
 * BF16 hi/lo operands, three products each (other precisions).  Start
 * (Section V, Texture Image Inpainting): l = u = 1, z = K l.
 *
 * cpa_completion_create: solver for m x n problems (m, n <= 65536, m n <=
 *   2^31) on the handle's device; owns 10 m n + m^2 + n^2 floats and about
 *   4 (m^2 + n^2 + 2 m n) BF16 values.
 * cpa_completion_run: dI device m x n (row stride ldi >= n), the observed
 *   values where dmask (uint8, row stride ldmask >= n) is nonzero, ignored
 *   elsewhere.  dL (row stride ldl >= n) receives the last least-squares
 *   iterate l; dZ1 (optional, contiguous m x n) the last shrinkage output.
 *   Outputs must not overlap the inputs or each other.  Runs max_iters
 *   iterations, or stops after the iteration whose E = |l_new - l|_F /
 *   |l_new|_F (the stopping quantity of the stopping-criterion footnote of Section V, Optimization Tools, computed
 *   after each least-squares step) is below tol > 0 (one host
 *   synchronisation per iteration).  *iters_done and errors (host, max_iters
 *   doubles) as for cpa_admm_rpca.  Errors: CPA_ERR_INVALID_ARG on bad
 *   arguments; errors of cpa_svt pass through. */
typedef struct cpa_completion_ctx *cpa_completion;
CPA_API cpa_status cpa_completion_create(cpa_handle h, int64_t m, int64_t n, cpa_completion *out);
CPA_API cpa_status cpa_completion_destroy(cpa_completion c);
CPA_API cpa_status cpa_completion_run(cpa_completion c, const float *dI, int64_t ldi, const uint8_t *dmask,
                                      int64_t ldmask, double tau_nuclear, double tau_l1, int L, int prec,
                                      int max_iters, double tol, float *dL, int64_t ldl, float *dZ1,
                                      int *iters_done, double *errors, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CPA_H */
