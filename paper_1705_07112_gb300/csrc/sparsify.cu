// Sparsity-based reduction of the filter (Section III-B, Eqs.
// sing_shrink_exact_sparse, threshold_components): the Gram matrix is
// rotated by an orthogonal (or masked) transform T, Phi = T G T^T, entries
// with |Phi_ij| < eps are set to zero, the Chebyshev filter is built on the
// thresholded Phi_, and the result is X T^T H_hat(Phi_) T.
//
// Transforms (p x p, row-major, FP32):
//   HAAR1_LOWPASS  one-level Haar DWT with the high band set to zero: row i
//                  < floor(p/2) holds 1/sqrt2 at columns 2i and 2i+1; for odd
//                  p row floor(p/2) holds 1 at column p-1; the rest are zero.
//   BLOCK_DCT8     block-diagonal orthonormal DCT-II with 8 x 8 blocks (the
//                  last block has size p mod 8 when that is not zero).
//   DCT            orthonormal DCT-II: T[k][j] = s_k cos(pi (2j+1) k / (2p)),
//                  s_0 = sqrt(1/p), s_k = sqrt(2/p).
// eps: given (mode ABS) or the k-th largest |Phi_ij|, k = ceil(frac p^2)
// clamped to [1, p^2] (mode TOPK, Eq. recommendation_epsilon's K(|Phi|, k));
// entries equal to eps are kept.
//
// Compaction.  Let S be the indices of the rows of Phi_ with a nonzero
// entry (s = |S|; Phi_ is symmetric, so its columns outside S are zero
// too).  After a permutation Phi_ = blockdiag(A, 0) with A = Phi_[S, S], so
// every polynomial of Phi_ -- each T_k(B_hat) and the truncated series H_hat
// -- is blockdiag(H_hat(A), c_out I) with c_out the series' value on the
// zero block: c_out = c_0 / 2 + sum_k c_k T_k(-sigma) (sigma = 1 on [0, b],
// (a + b) / (b - a) on the guarded interval).  The recurrence then runs on
// the s x s block A alone, and the filter applied to X is
//   T^T H T = T_S^T (H_hat(A) - c_out I) T_S + c_out T^T T
// with T_S the rows S of T (T^T T = I for the orthonormal transforms; for
// the masked Haar transform a 2 x 2 block-diagonal projection).  The power
// iteration on A from the start vector's entries at S gives the bound of
// Phi_ itself: every product with Phi_ is supported on S.
#include <algorithm>

#include "internal.h"

namespace cpa {
namespace {

__device__ double dct_entry(int size, int k, int j) {
    const double s = (k == 0) ? sqrt(1.0 / size) : sqrt(2.0 / size);
    return s * cospi((2.0 * j + 1.0) * k / (2.0 * size));
}

// cos(pi n / (2 p)), n = 0 .. 4p - 1 (FP64, rounded to FP32): every entry
// of the p x p DCT-II is s_k times one of them, n = (2j + 1) k mod 4p.
__global__ void dct_table_kernel(int p, float *tab) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < 4 * p; n += gridDim.x * blockDim.x)
        tab[n] = (float)cospi((double)n / (2.0 * p));
}

__global__ void make_transform_kernel(int type, int p, float *T, int64_t ld, const float *__restrict__ dct_tab) {
    const int64_t total = (int64_t)p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / p), j = (int)(e % p);
        double v = 0.0;
        if (type == CPA_T_IDENTITY) {
            v = (i == j) ? 1.0 : 0.0;
        } else if (type == CPA_T_HAAR1_LOWPASS) {
            const int h = p / 2;
            if (i < h) v = (j == 2 * i || j == 2 * i + 1) ? 0.70710678118654752440 : 0.0;
            else if ((p & 1) && i == h) v = (j == p - 1) ? 1.0 : 0.0;
        } else if (type == CPA_T_BLOCK_DCT8) {
            const int b = i / 8;
            if (j / 8 == b) {
                const int size = std::min(8, p - 8 * b);
                v = dct_entry(size, i - 8 * b, j - 8 * b);
            }
        } else {
            // s_k cos(pi (2j + 1) k / 2p) from the table (exact index arithmetic)
            const int64_t n = ((int64_t)(2 * j + 1) * i) % (4 * (int64_t)p);
            const float sk = i == 0 ? (float)sqrt(1.0 / p) : (float)sqrt(2.0 / p);
            T[(int64_t)i * ld + j] = sk * __ldg(dct_tab + n);
            continue;
        }
        T[(int64_t)i * ld + j] = (float)v;
    }
}

// Entries below eps set to zero; removed2 (optional) accumulates the sum of
// their squares, |Phi - Phi_|_F^2 (per-warp FP32 partials, FP64 atomics).
__global__ void threshold_kernel(float *Phi, int p, int64_t ld, const float *eps_dev, float eps_host,
                                 double *removed2, int *row_flags) {
    const float eps = eps_dev ? *eps_dev : eps_host;
    const int64_t total = (int64_t)p * p;
    float r2 = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / p;
        float *q = Phi + i * ld + e % p;
        const float v = *q;
        if (!(fabsf(v) >= eps)) {
            r2 = fmaf(v, v, r2);
            *q = 0.f;
        } else if (row_flags && v != 0.f) {
            row_flags[i] = 1;   // row i keeps a nonzero entry (same value from every writer)
        }
    }
    if (removed2) {
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        if ((threadIdx.x & 31) == 0 && r2 != 0.f) atomicAdd(removed2, (double)r2);
    }
}

// Full symmetric matrix from its lower triangle (row >= col valid).
__global__ void symmetrize_lower_kernel(float *S, int p, int64_t ld) {
    const int64_t total = (int64_t)p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / p), j = (int)(e % p);
        if (j > i) S[(int64_t)i * ld + j] = S[(int64_t)j * ld + i];
    }
}

// eps = k-th largest |Phi_ij| by a radix select over the IEEE bit patterns
// of |Phi| (order-preserving for non-negative floats), most significant
// digit first: bits 30..23, 22..15, 14..7, 6..0.  Each pass histograms the
// digit of the entries that match the digits chosen so far (per-block
// shared-memory histogram, added into global counts), then every block
// picks, from the top bin down, the bin holding the remaining rank.  One
// cooperative launch; a bounded grid barrier per pass.
__device__ __forceinline__ void grid_sync_sp(unsigned int *count, unsigned int &target, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        const long long t0 = clock64();
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > 4000000000LL) {
                atomicExch(err, (int)CPA_ERR_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();
}

constexpr int kTopkPasses = 4;
__device__ __constant__ int kTopkShift[kTopkPasses] = {23, 15, 7, 0};
__device__ __constant__ int kTopkBits[kTopkPasses] = {8, 8, 8, 7};

__global__ void __launch_bounds__(256) topk_eps_kernel(const float *__restrict__ Phi, int p, int64_t ld, long long k,
                                                       unsigned long long *counts /*[4][256]*/, unsigned int *bar,
                                                       int *err, float *eps_out) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned int sel_prefix;
    __shared__ unsigned long long sel_rank;
    unsigned int target = 0;
    unsigned int prefix = 0, pmask = 0;
    unsigned long long rank = (unsigned long long)k;   // rank among the entries matching prefix
    const int64_t total = (int64_t)p * p;
    for (int pass = 0; pass < kTopkPasses; ++pass) {
        const int sh = kTopkShift[pass];
        const unsigned int dmask = (1u << kTopkBits[pass]) - 1u;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        // warp-uniform trip count; lanes with equal bins add once (most
        // entries share a few exponent bins in the first pass)
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t first = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31);
        for (int64_t e0 = first; e0 < total; e0 += stride) {
            const int64_t e = e0 + (threadIdx.x & 31);
            int bin = -1;
            if (e < total) {
                const unsigned int b = __float_as_uint(fabsf(__ldg(Phi + (e / p) * ld + e % p)));
                if ((b & pmask) == prefix) bin = (int)((b >> sh) & dmask);
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, bin);
            if (bin >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned int)__popc(peers));
        }
        __syncthreads();
        unsigned long long *cnt = counts + pass * 256;
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            if (hist[i]) atomicAdd(&cnt[i], (unsigned long long)hist[i]);
        grid_sync_sp(bar, target, err);
        if (threadIdx.x == 0) {
            // the bin of the rank-th largest entry: from the top bin down
            unsigned long long above = 0;
            int j = (int)dmask;
            for (; j > 0; --j) {
                const unsigned long long c = __ldcg(&cnt[j]);
                if (above + c >= rank) break;
                above += c;
            }
            sel_prefix = (unsigned int)j;
            sel_rank = rank - above;
        }
        __syncthreads();
        prefix |= sel_prefix << sh;
        pmask |= dmask << sh;
        rank = sel_rank;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *eps_out = __uint_as_float(prefix);
}

// idx[0 .. s) = the flagged rows in ascending order, *s_out = s (one block).
__global__ void compact_kernel(const int *__restrict__ flags, int p, int *idx, int *s_out) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < p; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int f = i < p ? flags[i] : 0;
        const unsigned int bal = __ballot_sync(0xffffffffu, f);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int off = base;
        for (int w = 0; w < warp; ++w) off += warp_tot[w];
        if (f) idx[off + before] = i;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < nw; ++w) base += warp_tot[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *s_out = base;
}

// A[a][b] = Phi[idx[a]][idx[b]], a, b < s.
__global__ void gather_block_kernel(const float *__restrict__ Phi, int64_t ld, const int *__restrict__ idx, int s,
                                    float *A, int64_t lda) {
    const int64_t total = (int64_t)s * s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / s), b = (int)(e % s);
        A[(int64_t)a * lda + b] = Phi[(int64_t)__ldg(idx + a) * ld + __ldg(idx + b)];
    }
}

// R[a][j] = T[idx[a]][j], a < s, j < p.
__global__ void gather_rows_kernel(const float *__restrict__ T, int64_t ld, const int *__restrict__ idx, int s, int p,
                                   float *R, int64_t ldr) {
    const int64_t total = (int64_t)s * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / p), j = (int)(e % p);
        R[(int64_t)a * ldr + j] = T[(int64_t)__ldg(idx + a) * ld + j];
    }
}

// *c_out = c_0 / 2 + sum_{k=1}^{L-1} c_k T_k(-sigma) (FP64, the three-term
// recurrence of the Chebyshev polynomials at the scalar -sigma).
__global__ void zero_block_value_kernel(const double *__restrict__ c, int L, double sigma, double *c_out) {
    const double x = -sigma;
    double t0 = 1.0, t1 = x, v = 0.5 * c[0];
    if (L > 1) v += c[1] * t1;
    for (int k = 2; k < L; ++k) {
        const double t2 = 2.0 * x * t1 - t0;
        v += c[k] * t2;
        t0 = t1;
        t1 = t2;
    }
    *c_out = v;
}

// H[i][i] += scale * (*c), i < s (FP32 result).
__global__ void diag_add_kernel(float *H, int s, int64_t ld, const double *__restrict__ c, double scale) {
    const float v = (float)(scale * *c);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x) H[(int64_t)i * ld + i] += v;
}

// F += (*c) T^T T for the transform `type` (p x p): the identity for the
// orthonormal transforms; for the masked Haar transform 1/2 on each 2 x 2
// block of the pairs (2i, 2i + 1), i < floor(p/2), and 1 at (p-1, p-1) for
// odd p.
__global__ void add_transform_gram_kernel(float *F, int p, int64_t ld, int type, const double *__restrict__ c) {
    const float v = (float)*c;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x) {
        if (type != CPA_T_HAAR1_LOWPASS) {
            F[(int64_t)i * ld + i] += v;
        } else if ((p & 1) && i == p - 1) {
            F[(int64_t)i * ld + i] += v;
        } else {
            const int j = i ^ 1;   // the pair's other index
            F[(int64_t)i * ld + i] += 0.5f * v;
            F[(int64_t)i * ld + j] += 0.5f * v;
        }
    }
}

}  // namespace

cudaError_t compact_support(const int *flags, int p, int *idx, int *s_dev, cudaStream_t st) {
    compact_kernel<<<1, 1024, 0, st>>>(flags, p, idx, s_dev);
    return cudaGetLastError();
}

cudaError_t gather_block(const float *Phi, int64_t ld, const int *idx, int s, float *A, int64_t lda, cudaStream_t st,
                         int num_sms) {
    const int64_t total = (int64_t)s * s;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8));
    gather_block_kernel<<<blocks, 256, 0, st>>>(Phi, ld, idx, s, A, lda);
    return cudaGetLastError();
}

cudaError_t gather_rows(const float *T, int64_t ld, const int *idx, int s, int p, float *R, int64_t ldr,
                        cudaStream_t st, int num_sms) {
    const int64_t total = (int64_t)s * p;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8));
    gather_rows_kernel<<<blocks, 256, 0, st>>>(T, ld, idx, s, p, R, ldr);
    return cudaGetLastError();
}

cudaError_t zero_block_value(const double *c, int L, double sigma, double *c_out, cudaStream_t st) {
    zero_block_value_kernel<<<1, 1, 0, st>>>(c, L, sigma, c_out);
    return cudaGetLastError();
}

cudaError_t diag_add(float *H, int s, int64_t ld, const double *c, double scale, cudaStream_t st) {
    diag_add_kernel<<<std::max(1, std::min((s + 255) / 256, 64)), 256, 0, st>>>(H, s, ld, c, scale);
    return cudaGetLastError();
}

cudaError_t add_transform_gram(float *F, int p, int64_t ld, int type, const double *c, cudaStream_t st) {
    add_transform_gram_kernel<<<std::max(1, std::min((p + 255) / 256, 64)), 256, 0, st>>>(F, p, ld, type, c);
    return cudaGetLastError();
}

cudaError_t make_transform(int type, int p, float *T, int64_t ld, cudaStream_t st, int num_sms, float *scratch) {
    const int64_t total = (int64_t)p * p;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    if (type == CPA_T_DCT) {
        if (!scratch) return cudaErrorInvalidValue;
        dct_table_kernel<<<std::max(1, std::min((4 * p + 255) / 256, num_sms * 4)), 256, 0, st>>>(p, scratch);
    }
    make_transform_kernel<<<std::max(blocks, 1), 256, 0, st>>>(type, p, T, ld, scratch);
    return cudaGetLastError();
}

cudaError_t threshold_entries(float *Phi, int p, int64_t ld, const float *eps_dev, float eps_host, cudaStream_t st,
                              int num_sms, double *removed2, int *row_flags) {
    const int64_t total = (int64_t)p * p;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    if (row_flags) {
        cudaError_t r = cudaMemsetAsync(row_flags, 0, sizeof(int) * (size_t)p, st);
        if (r != cudaSuccess) return r;
    }
    threshold_kernel<<<std::max(blocks, 1), 256, 0, st>>>(Phi, p, ld, eps_dev, eps_host, removed2, row_flags);
    return cudaGetLastError();
}

cudaError_t symmetrize_lower(float *S, int p, int64_t ld, cudaStream_t st, int num_sms) {
    const int64_t total = (int64_t)p * p;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    symmetrize_lower_kernel<<<std::max(blocks, 1), 256, 0, st>>>(S, p, ld);
    return cudaGetLastError();
}

cudaError_t topk_eps(const float *Phi, int p, int64_t ld, long long k, unsigned long long *counts, unsigned int *bar,
                     int *err, float *eps_out, cudaStream_t st, int num_sms) {
    cudaError_t r = cudaMemsetAsync(counts, 0, kTopkCounts * sizeof(unsigned long long), st);
    if (r == cudaSuccess) r = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
    if (r == cudaSuccess) r = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (r != cudaSuccess) return r;
    const int64_t total = (int64_t)p * p;
    int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms);
    grid = std::max(grid, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, topk_eps_kernel, Phi, p, ld, k, counts, bar, err, eps_out);
}

}  // namespace cpa
