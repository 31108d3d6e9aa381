// Batched CPA shrinkage of many small matrices (patch groups), one
// persistent launch.
//
// One CTA of 128 threads (4 warps) owns one matrix at a time and walks a
// size-sorted work list.  With p = min(m, n) <= 64 and q = max(m, n) <= 128
// everything stays on chip:
//   shared memory  X as BF16 hi/lo (or FP32), At = (2/lambda) G as BF16 hi/lo
//                  (the constant operand), Psi_{k-1} as BF16 hi/lo (double
//                  buffered), G in FP32 for the power iteration;
//   registers      the accumulator and Psi_{k-1}, Psi_{k-2}, H in the MMA
//                  accumulator layout: warp w owns rows 16w..16w+15, each
//                  thread the same 32 elements at every step, so the
//                  recurrence  Psi_k = 2 At Psi_{k-1} - 2 Psi_{k-1} - Psi_{k-2},
//                  H += c_k Psi_k  never leaves the registers.
// Products (Gram, recurrence, final product) use warp-level BF16 tensor-core
// MMA (m16n8k16, FP32 accumulate) with the hi/lo split hi*hi + hi*lo + lo*hi,
// or FP32 FMA in the plain-FP32 variant.  The 64 x 64 products of this
// workload are too small for a 128-row tcgen05 tile to pay for its TMEM round
// trips; the path is bound by the per-element recurrence arithmetic.
//
// The recurrence multiplies At by Psi_{k-1} exactly as stored (B operand
// loaded with a transposing ldmatrix from row-major Psi), so no symmetry of
// Psi is assumed.  Lambda_max, the coefficients and everything else follow
// the single-matrix path's definitions.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace cpa {
namespace {

constexpr int kP = 64;          // maximum min(m, n)
constexpr int kQ = 128;         // maximum max(m, n)
constexpr int kLdB = kP + 8;    // BF16 row stride of 64-wide tiles (conflict-free ldmatrix)
constexpr int kLdX = kQ + 8;    // BF16 row stride of X tiles
constexpr int kThreads = 128;
constexpr int kMaxBatchTerms = 1024;
constexpr uint64_t kEdgeSeedXor = 0x5EEDULL;   // start vector of the lower-edge feature


// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t su32b(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(su32b(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(su32b(p)));
}

__device__ __forceinline__ void mma_bf16_16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---------------------------------------------------------------- fragments
//
// Accumulator layout of m16n8k16 (per warp: 16 rows x 64 columns = 8 n-tiles):
// thread (g = lane/4, t = lane%4) holds for n-tile nt the elements
//   (16w + g,     8 nt + 2t + {0,1})  -> d[nt][0..1]
//   (16w + g + 8, 8 nt + 2t + {0,1})  -> d[nt][2..3]

struct Frag {
    float v[8][4];
};

__device__ __forceinline__ void frag_zero(Frag &f) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) f.v[a][b] = 0.f;
}

__device__ __forceinline__ int frag_row(int w, int lane, int e) { return 16 * w + (lane >> 2) + (e >= 2 ? 8 : 0); }
__device__ __forceinline__ int frag_col(int nt, int lane, int e) { return 8 * nt + 2 * (lane & 3) + (e & 1); }

// A fragment (16 rows from r0, 16 columns from k0) of a row-major BF16 tile.
__device__ __forceinline__ void load_a(uint32_t *a, const __nv_bfloat16 *base, int ld, int r0, int k0, int lane) {
    const __nv_bfloat16 *p = base + (r0 + (lane & 15)) * ld + k0 + (lane >> 4) * 8;
    ldsm_x4(a[0], a[1], a[2], a[3], p);
}
// A fragment of A = S^T where S is a row-major BF16 tile (A(i,k) = S(k,i)).
__device__ __forceinline__ void load_a_t(uint32_t *a, const __nv_bfloat16 *base, int ld, int r0, int k0, int lane) {
    // matrices: a0 = S[k0..+7][r0..+7]^T, a1 = S[k0..+7][r0+8..]^T, a2 = S[k0+8..][r0..]^T, a3 = S[k0+8..][r0+8..]^T
    const int mtx = lane >> 3, r = lane & 7;
    const int kk = k0 + ((mtx & 2) ? 8 : 0) + r;
    const int ii = r0 + ((mtx & 1) ? 8 : 0);
    ldsm_x4_t(a[0], a[1], a[2], a[3], base + kk * ld + ii);
}
// B fragments for two n-tiles (columns n0..n0+15), k from k0, of B(k,j) stored
// row-major as S[k][j] (transposing load).  b[0],b[1]: n-tile n0; b[2],b[3]: n0+8.
__device__ __forceinline__ void load_b_kn(uint32_t *b, const __nv_bfloat16 *base, int ld, int k0, int n0, int lane) {
    const int mtx = lane >> 3, r = lane & 7;
    const int kk = k0 + ((mtx & 1) ? 8 : 0) + r;
    const int jj = n0 + ((mtx & 2) ? 8 : 0);
    ldsm_x4_t(b[0], b[1], b[2], b[3], base + kk * ld + jj);
}
// B fragments of B(k,j) stored as S[j][k] (non-transposing load).
__device__ __forceinline__ void load_b_nk(uint32_t *b, const __nv_bfloat16 *base, int ld, int k0, int n0, int lane) {
    const int mtx = lane >> 3, r = lane & 7;
    const int jj = n0 + ((mtx & 2) ? 8 : 0) + r;
    const int kk = k0 + ((mtx & 1) ? 8 : 0);
    ldsm_x4(b[0], b[1], b[2], b[3], base + jj * ld + kk);
}

// ---------------------------------------------------------------- shared memory

struct BatchSmem {
    __nv_bfloat16 xhi[kP * kLdX];        // Xp = X^T (m >= n) or X (m < n): p x q, hi
    __nv_bfloat16 xlo[kP * kLdX];
    __nv_bfloat16 ahi[kP * kLdB];        // At = (2/lambda) G
    __nv_bfloat16 alo[kP * kLdB];
    __nv_bfloat16 zhi[2][kP * kLdB];     // Psi_{k-1}, double buffered
    __nv_bfloat16 zlo[2][kP * kLdB];
    float g[kP * (kP + 1)];              // G (FP32), then H for the final product
    float v[2][kP];                      // power-iteration vectors
    float redf[8];                       // bsumf partials, two sets of four
    float coef[kMaxBatchTerms];          // c_k (summed in FP64, kept in FP32: the recurrence's epilogue
                                         // arithmetic); before that, the predictor's scratch
    double scal[4];                      // theta, r, trace, lambda
    double lam;                          // the bound, formed by thread 0
    float s2;                            // 2 / lambda in FP32, formed by thread 0
    int next_it;                         // work item fetched by thread 0
};

// The coefficient sums' FP64 scratch, in the Psi_{k-1} buffers' lo halves
// (free until the shift): a table of cos(pi m / 2L) for m = 0..L and the
// response at the L nodes, 2L + 1 doubles.
static_assert((2 * kMaxBatchTerms + 1) * sizeof(double) <= 2 * kP * kLdB * sizeof(__nv_bfloat16),
              "coefficient scratch");
__device__ __forceinline__ double *coef_tab(BatchSmem &S) { return reinterpret_cast<double *>(&S.zlo[0][0]); }

// cos(pi m / 2L) for any integer m >= 0 from the table of m = 0..L:
// cos(2 pi - x) = cos x and cos(pi - x) = -cos x.
__device__ __forceinline__ double cos_from_tab(const double *tab, int m, int L) {
    m %= 4 * L;
    if (m > 2 * L) m = 4 * L - m;
    return m > L ? -tab[2 * L - m] : tab[m];
}

// Block sum (4 warps) of one float per thread.  The warp partials go through
// one of two sets of shared slots, alternating with `slot`, so one barrier
// per call suffices: a set is rewritten two calls later, after every thread
// has passed the barrier of the call in between (and so has read it).
__device__ __forceinline__ float bsumf(float x, float *red8, int &slot) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    float *r = red8 + 4 * (slot & 1);
    ++slot;
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = x;
    __syncthreads();
    return (r[0] + r[1]) + (r[2] + r[3]);
}

// (G v)(row) from the FP32 Gram matrix in shared memory: two threads per row
// (half = 0, 1 take alternate columns), two accumulators each; rows >= p
// give 0.  Called by all threads of the block (pair shuffle).
__device__ __forceinline__ float gmatvec(const BatchSmem &S, int row, int half, int p, const float *v) {
    float a0 = 0.f, a1 = 0.f;
    if (row < p) {
        const float *gr = S.g + row * (kP + 1);
        int j = half;
        for (; j + 2 < p; j += 4) {
            a0 = fmaf(gr[j], v[j], a0);
            a1 = fmaf(gr[j + 2], v[j + 2], a1);
        }
        if (j < p) a0 = fmaf(gr[j], v[j], a0);
    }
    const float a = a0 + a1;
    return a + __shfl_xor_sync(0xffffffffu, a, 1);
}

__device__ __forceinline__ uint64_t splitmix64_b(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// D(16w.., 0..63) = sum_k A(i,k) B(k,j) over K (multiple of 16, <= kQ),
// hi/lo split when split.  a_trans: A = S^T of a row-major S[k][i];
// b_kn: B stored S[k][j], else S[j][k].
template <bool A_T, bool B_KN>
__device__ __forceinline__ void mma_tile(Frag &d, const __nv_bfloat16 *ahi, const __nv_bfloat16 *alo, int lda,
                                         const __nv_bfloat16 *bhi, const __nv_bfloat16 *blo, int ldb, int K,
                                         bool split, int w, int lane) {
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t ah[4], al[4];
        if (A_T) {
            load_a_t(ah, ahi, lda, 16 * w, k0, lane);
            if (split) load_a_t(al, alo, lda, 16 * w, k0, lane);
        } else {
            load_a(ah, ahi, lda, 16 * w, k0, lane);
            if (split) load_a(al, alo, lda, 16 * w, k0, lane);
        }
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t bh[4], bl[4];
            if (B_KN) {
                load_b_kn(bh, bhi, ldb, k0, 16 * np, lane);
                if (split) load_b_kn(bl, blo, ldb, k0, 16 * np, lane);
            } else {
                load_b_nk(bh, bhi, ldb, k0, 16 * np, lane);
                if (split) load_b_nk(bl, blo, ldb, k0, 16 * np, lane);
            }
            mma_bf16_16816(d.v[2 * np], ah, bh[0], bh[1]);
            mma_bf16_16816(d.v[2 * np + 1], ah, bh[2], bh[3]);
            if (split) {
                mma_bf16_16816(d.v[2 * np], ah, bl[0], bl[1]);
                mma_bf16_16816(d.v[2 * np + 1], ah, bl[2], bl[3]);
                mma_bf16_16816(d.v[2 * np], al, bh[0], bh[1]);
                mma_bf16_16816(d.v[2 * np + 1], al, bh[2], bh[3]);
            }
        }
    }
}

__device__ __forceinline__ void put_hilo(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int idx, float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Writes a fragment (rows 16w..+15, columns 0..63) to a row-major BF16
// hi/lo tile.
__device__ __forceinline__ void frag_store_hilo(const Frag &f, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int ld, int w,
                                                int lane) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int r = frag_row(w, lane, 2 * h2), c = frag_col(nt, lane, 0);
            const float x0 = f.v[nt][2 * h2], x1 = f.v[nt][2 * h2 + 1];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            *reinterpret_cast<uint32_t *>(hi + r * ld + c) = pack2(h0, h1);
            *reinterpret_cast<uint32_t *>(lo + r * ld + c) = pack2(l0, l1);
        }
    }
}

// FP32 FMA product for the plain variant: D(16w.., 0..63) += sum_k A(i,k) B(k,j)
// with A, B given as FP32 element accessors through shared memory.
template <class FA, class FB>
__device__ __forceinline__ void fma_tile(Frag &d, FA A, FB B, int K, int w, int lane) {
    for (int k = 0; k < K; ++k) {
        float a0 = A(frag_row(w, lane, 0), k), a1 = A(frag_row(w, lane, 2), k);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float b0 = B(k, frag_col(nt, lane, 0)), b1 = B(k, frag_col(nt, lane, 1));
            d.v[nt][0] = fmaf(a0, b0, d.v[nt][0]);
            d.v[nt][1] = fmaf(a0, b1, d.v[nt][1]);
            d.v[nt][2] = fmaf(a1, b0, d.v[nt][2]);
            d.v[nt][3] = fmaf(a1, b1, d.v[nt][3]);
        }
    }
}

// FP32 variant: Psi buffer b spans zhi[0..1] (b = 0) or zlo[0..1] (b = 1).
__device__ __forceinline__ float *zbuf_f32(BatchSmem &S, int b) {
    return reinterpret_cast<float *>(b == 0 ? &S.zhi[0][0] : &S.zlo[0][0]);
}

// ---------------------------------------------------------------- the kernel
//
// FP32 variant: the BF16 buffers are reused as FP32 storage (xhi/xlo hold X
// in FP32, ahi/alo hold At, zhi[b]/zlo[b] hold Psi_{k-1}).

// Feature vector of one matrix for the learned predictor (kFeatures
// entries, defined in the declaration of cpa_batch_features): shape, energy
// and threshold relative to theta_4 (a lower bound of Lambda_max after four
// power products), the lower spectral edge, |G|_F^2, convergence of the
// power iterates, and the shrink kind.
constexpr int kFeatures = 12;
constexpr int kHidden = 64;   // the predictor network: kFeatures -> 64 -> 64 -> 2


// Features of one matrix (FEAT: written out, returns L = -1) or the learned
// choice of (Lambda_max, L) for it (LEARN).  Kept out of line so that the
// recurrence of the calling kernel is compiled as in the plain mode.
struct Choice {
    double lam;
    int L;
};

template <bool FEAT>
__device__ __noinline__ Choice learned_phase(BatchSmem &S, int idx, int p, int q, ShrinkParams sp, float th2, float th4,
                                             float r4, double lam, float *__restrict__ feat,
                                             double *__restrict__ theta_out, const LearnArgs la) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int row = tid >> 1, half = tid & 1;
    const bool own = row < p && half == 0;
    int rs = 0;   // a barrier precedes the first reduction
        // lower spectral edge: 4 steps u <- (theta4 I - G) u / |.| from a
        // second SplitMix64 vector, then lambda_min = u^T G u / u^T u
        __syncthreads();
        for (int i = tid; i < p; i += kThreads) {
            const uint64_t z = splitmix64_b(kStartSeed ^ kEdgeSeedXor, (uint64_t)i);
            S.v[0][i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
        }
        __syncthreads();
        float lmin = 0.f;
        int uc = 0;
        for (int t = 0; t <= 4; ++t) {
            const float a = gmatvec(S, row, half, p, S.v[uc]);
            const float ur = own ? S.v[uc][row] : 0.f;
            if (t < 4) {
                const float nx = th4 * ur - a;
                const float n2 = bsumf(own ? nx * nx : 0.f, S.redf, rs);
                const float sc2 = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
                if (own) S.v[uc ^ 1][row] = nx * sc2;
                __syncthreads();
                uc ^= 1;
            } else {
                const float num = bsumf(ur * a, S.redf, rs);
                const float den = bsumf(ur * ur, S.redf, rs);
                lmin = den > 0.f ? num / den : 0.f;
            }
        }
        float fro = 0.f;
        for (int r = w; r < p; r += kThreads / 32)
            for (int c = lane; c < p; c += 32) {
                const float gv = S.g[r * (kP + 1) + c];
                fro = fmaf(gv, gv, fro);
            }
        fro = bsumf(fro, S.redf, rs);
        const float tr = bsumf(own ? S.g[row * (kP + 1) + row] : 0.f, S.redf, rs);
        // one feature per thread (threads 0..11): ratio in FP64, log in FP32
        float *fv = S.coef;   // free until the coefficients are formed
        if (tid < kFeatures) {
            const double tiny = 1e-30;
            const double E = tr > 0.f ? (double)tr : 1.0;
            const double t4 = fmax((double)th4, tiny * E);
            double thr2;   // squared threshold on sigma (weighted soft: its level at theta4)
            if (sp.kind == CPA_WSOFT) {
                const double se = sqrt(fmax((double)th4 - sp.noise, 0.0));
                const double wv = sp.c / (se + sp.eps);
                thr2 = wv * wv;
            } else {
                thr2 = sp.tau * sp.tau;
            }
            thr2 = fmax(thr2, tiny * E);
            const double lm = fmax((double)lmin, tiny * E);
            double r = 1.0;
            switch (tid) {
                case 0: r = (double)p; break;
                case 1: r = (double)q / (double)p; break;
                case 2: r = E / t4; break;
                case 3: r = thr2 / t4; break;
                case 4: r = lm / t4; break;
                case 5: r = thr2 / lm; break;
                case 6: r = fmax((double)fro, tiny * E * E) / (t4 * t4); break;
                case 7: r = E / ((double)p * thr2); break;
                case 8: r = t4 / fmax((double)th2, tiny * E); break;
                case 9: r = (t4 + (double)r4) / t4; break;
                default: break;
            }
            fv[tid] = tid == 10 ? (sp.kind == CPA_HARD ? 1.f : 0.f)
                      : tid == 11 ? (sp.kind == CPA_WSOFT ? 1.f : 0.f)
                                  : logf((float)r);
        }
        if (FEAT) {
            __syncthreads();
            if (tid < kFeatures) feat[(int64_t)idx * kFeatures + tid] = fv[tid];
            if (tid == 0) theta_out[idx] = (double)th4;
            __syncthreads();
            return Choice{0.0, -1};
        }
        // network forward.  The weights are staged in shared memory (the
        // recurrence buffers, free until the shift) with padded rows
        // (W1 stride 13, W2 stride 65: conflict-free), then one output per
        // thread in the summation order of the network's own forward
        // kernel (same FP32 results).
        constexpr int ob1 = kHidden * kFeatures, oW2 = ob1 + kHidden, ob2 = oW2 + kHidden * kHidden,
                      oW3 = ob2 + kHidden, ob3 = oW3 + 2 * kHidden, nP = ob3 + 2;
        constexpr int sW1 = 0, sb1 = kHidden * (kFeatures + 1), sW2 = sb1 + kHidden,
                      sb2 = sW2 + kHidden * (kHidden + 1), sW3 = sb2 + kHidden, sb3 = sW3 + 2 * kHidden;
        static_assert((sb3 + 2) * sizeof(float) <= sizeof(S.zhi) + sizeof(S.zlo), "staged network");
        float *wsm = reinterpret_cast<float *>(S.zhi);
        auto staged = [&](int e) {   // shared-memory position of parameter e
            if (e < ob1) return sW1 + (e / kFeatures) * (kFeatures + 1) + e % kFeatures;
            if (e < oW2) return sb1 + (e - ob1);
            if (e < ob2) return sW2 + ((e - oW2) / kHidden) * (kHidden + 1) + (e - oW2) % kHidden;
            return sb2 + (e - ob2);   // b2, W3, b3 keep their relative layout
        };
        {
            // all loads first (16-byte, coalesced), then the scatter
            constexpr int n4 = nP / 4, per = (n4 + kThreads - 1) / kThreads;
            const float4 *P4 = reinterpret_cast<const float4 *>(la.P);
            float4 buf[per];
#pragma unroll
            for (int k = 0; k < per; ++k) {
                const int e4 = tid + k * kThreads;
                if (e4 < n4) buf[k] = __ldg(P4 + e4);
            }
#pragma unroll
            for (int k = 0; k < per; ++k) {
                const int e4 = tid + k * kThreads;
                if (e4 < n4) {
                    wsm[staged(4 * e4)] = buf[k].x;
                    wsm[staged(4 * e4 + 1)] = buf[k].y;
                    wsm[staged(4 * e4 + 2)] = buf[k].z;
                    wsm[staged(4 * e4 + 3)] = buf[k].w;
                }
            }
            if (tid < nP - 4 * n4) wsm[staged(4 * n4 + tid)] = __ldg(la.P + 4 * n4 + tid);
        }
        __syncthreads();
        float *h1 = fv + 16, *h2 = h1 + kHidden, *yv = h2 + kHidden;
        if (tid < kHidden) {
            float a = wsm[sb1 + tid];
            for (int j = 0; j < kFeatures; ++j) a = fmaf(wsm[sW1 + tid * (kFeatures + 1) + j], fv[j], a);
            h1[tid] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (tid < kHidden) {
            float a = wsm[sb2 + tid];
            for (int j = 0; j < kHidden; ++j) a = fmaf(wsm[sW2 + tid * (kHidden + 1) + j], h1[j], a);
            h2[tid] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (tid < 2) {
            float a = wsm[sb3 + tid];
            for (int j = 0; j < kHidden; ++j) a = fmaf(wsm[sW3 + tid * kHidden + j], h2[j], a);
            yv[tid] = a;
        }
        __syncthreads();
        // decision rule, taken by thread 0 and broadcast.  The predicted
        // bound is never taken below the residual-corrected estimate
        // (theta_4 + r_4)(1 + 0.01): below sigma_max^2 the series grows
        // outside [-1, 1]
        if (tid == 0) {
            const double y0 = (double)yv[0], y1 = (double)yv[1];
            const double Lf = ceil(exp(y1) * la.L_scale);
            const bool ok_L = isfinite(Lf) && Lf <= (double)la.L_max;
            int Lc = ok_L ? (int)Lf : la.L_fallback;
            if (Lc < la.L_min) Lc = la.L_min;
            double lc = lam;
            bool ok_lam = true;
            if (la.use_lambda) {
                const double lp = (double)th4 * exp(fmax(y0, 0.0)) * (1.0 + la.margin);
                const double floor_lam = ((double)th4 + (double)r4) * (1.0 + kLambdaMargin);
                ok_lam = isfinite(lp) && lp > 0.0;
                if (isfinite(lp) && lp > 0.0) {
                    lc = fmax(lp, floor_lam);
                } else {
                    Lc = la.L_fallback;   // non-finite prediction: the bound and the fallback order
                }
            }
            la.L_out[idx] = Lc;
            if (!ok_L || !ok_lam) atomicAdd(la.nfallback, 1);
            S.scal[0] = lc;
            S.next_it = Lc;   // free until the next fetch
        }
        __syncthreads();
        const Choice c{S.scal[0], S.next_it};
        __syncthreads();   // S.coef and S.next_it are rewritten by the caller
        return c;
}

// Modes: FEAT writes the features (and theta_4) and stops; LEARN computes
// them, runs the network and the decision rule, then shrinks with the
// chosen (Lambda_max, L); neither: plain shrinkage.
template <bool TC, bool FEAT, bool LEARN>
__global__ void __launch_bounds__(kThreads, 2)
    batched_kernel(const BatchDesc *__restrict__ descs, const int *__restrict__ order, int count,
                   const float *__restrict__ X, float *__restrict__ Y, const ShrinkParams *__restrict__ shr,
                   int shr_stride, const double *__restrict__ lam_in, double *__restrict__ lam_out, int iters,
                   int *__restrict__ status, const int *__restrict__ L_in, float *__restrict__ feat,
                   double *__restrict__ theta_out, const LearnArgs la) {
    extern __shared__ __align__(16) uint8_t smem_raw_b[];
    BatchSmem &S = *reinterpret_cast<BatchSmem *>(smem_raw_b);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;

    // dynamic work list: each CTA fetches its next matrix from a counter
    // (status[1], zero at launch), so CTAs that drew cheap matrices take
    // more of them; matrices are listed largest estimated work first
    for (;;) {
        if (tid == 0) S.next_it = atomicAdd(status + 1, 1);
        __syncthreads();
        const int it = S.next_it;
        if (it >= count) break;
        const int idx = order[it];
        const BatchDesc d = descs[idx];
        const int m = d.m, n = d.n;
        int L = L_in ? L_in[idx] : d.L;
        const bool tall = m >= n;           // Gram X^T X (p = n) or X X^T (p = m)
        const int p = tall ? n : m, q = tall ? m : n;
        const int q16 = (q + 15) & ~15, p16 = (p + 15) & ~15;
        const float *Xg = d.x ? d.x : X + d.off;
        float *Yg = d.x ? d.y : Y + d.off;
        const int64_t ldxm = d.x ? d.ldx : n, ldym = d.x ? d.ldy : n;
        const ShrinkParams sp = shr[shr_stride ? idx : 0];

        // ---- Xp (p x q, zero padded to multiples of 16) into shared memory:
        // Xp = X^T when m >= n, else X, so that G = Xp Xp^T and the final
        // product is H Xp (stored back transposed when m >= n).  X is read
        // in its own row-major order (coalesced), sixteen independent loads
        // in flight per thread, then scattered; the padding is zeroed apart.
        {
            auto put = [&](int idx, float x) {
                if (TC)
                    put_hilo(S.xhi, S.xlo, idx, x);
                else
                    reinterpret_cast<float *>(S.xhi)[idx] = x;   // spans xhi and xlo
            };
            for (int e = tid; e < p16 * q16; e += kThreads) {
                const int r = e / q16, c = e - r * q16;
                if (r >= p || c >= q) put(r * kLdX + c, 0.f);
            }
            const int mn = m * n;
            for (int base = 0; base < mn; base += 16 * kThreads) {
                float v[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int e = base + k * kThreads + tid;
                    const int i = e / n, j = e - i * n;
                    v[k] = e < mn ? __ldg(Xg + (int64_t)i * ldxm + j) : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int e = base + k * kThreads + tid;
                    if (e < mn) {
                        const int i = e / n, j = e - i * n;
                        put(tall ? j * kLdX + i : i * kLdX + j, v[k]);
                    }
                }
            }
        }
        __syncthreads();

        // ---- Gram G(i,j) = sum_k Xp(i,k) Xp(j,k) (FP32 accumulate), into S.g
        Frag acc;
        frag_zero(acc);
        if (TC) {
            mma_tile<false, false>(acc, S.xhi, S.xlo, kLdX, S.xhi, S.xlo, kLdX, q16, true, w, lane);
        } else {
            const float *xf = reinterpret_cast<const float *>(S.xhi);
            fma_tile(acc, [&](int i, int k) { return xf[i * kLdX + k]; },
                     [&](int k, int j) { return xf[j * kLdX + k]; }, q, w, lane);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                S.g[frag_row(w, lane, e) * (kP + 1) + frag_col(nt, lane, e)] = acc.v[nt][e];
        __syncthreads();

        // ---- Lambda_max: power iteration (definition of cpa_lambda_bound)
        double lam = lam_in ? lam_in[idx] : 0.0;
        float th2 = 0.f, th4 = 0.f, r4 = 0.f;   // features: theta_2, theta_4, residual after 4 products
        int rs = 0;                             // reduction slot parity (bsumf)
        const int row = tid >> 1, half = tid & 1;
        const bool own = row < p && half == 0;  // the thread that keeps row `row` of a vector
        if (!(lam > 0.0) || FEAT || LEARN) {
            float s0 = 0.f;
            for (int i = tid; i < p; i += kThreads) {
                const uint64_t z = splitmix64_b(kStartSeed, (uint64_t)i);
                const float x = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
                S.v[0][i] = x;
                s0 = fmaf(x, x, s0);
            }
            float nrm2 = bsumf(s0, S.redf, rs);
            int cur = 0;
            // the learned choice with the predicted bound needs only the
            // features' four products; its fallback bound is theirs
            const int its = (FEAT || (LEARN && la.use_lambda)) ? 4 : iters;
            for (int t = 0; t <= its; ++t) {
                // w = G (v / |v|): two threads per row
                const float sc = nrm2 > 0.f ? 1.f / sqrtf(nrm2) : 0.f;
                const float a = gmatvec(S, row, half, p, S.v[cur]) * sc;
                const float vt = own ? S.v[cur][row] : 0.f;
                if (own) S.v[cur ^ 1][row] = a;
                if ((FEAT || LEARN) && t < its && t < 4) {
                    // theta after t+1 products: (v/|v|)^T G (v/|v|), v the input of this product
                    const float th = bsumf(vt * a, S.redf, rs) * sc;
                    if (t == 1) th2 = th;
                    if (t == 3) {
                        th4 = th;
                        const float dd = own ? a - th * vt * sc : 0.f;   // G v - theta v, v unit
                        r4 = sqrtf(fmaxf(bsumf(dd * dd, S.redf, rs), 0.f));
                    }
                }
                if (t < its) {
                    nrm2 = bsumf(own ? a * a : 0.f, S.redf, rs);
                    cur ^= 1;
                } else {
                    // v = S.v[cur] / |v| (unit), a = (G v)(row)
                    const float vu = vt * sc;
                    const float th = bsumf(vu * a, S.redf, rs);
                    const float dd = own ? a - th * vu : 0.f;
                    const float r2 = bsumf(dd * dd, S.redf, rs);
                    const float tr = bsumf(own ? S.g[row * (kP + 1) + row] : 0.f, S.redf, rs);
                    // one thread: FP64 square roots are long sequences on
                    // this part's scarce FP64 pipe
                    if (tid == 0) {
                        double lb = ((double)th + sqrt((double)fmaxf(r2, 0.f))) * (1.0 + kLambdaMargin);
                        if (lb > (double)tr) lb = (double)tr;
                        if (!isfinite(lb) || !isfinite(tr)) {
                            atomicExch(status, (int)CPA_ERR_NONFINITE);
                            lb = 1.0;
                        } else if (!(lb > 0.0)) {
                            lb = tr > 0.f ? (double)tr : 1.0;
                        }
                        S.lam = lb;
                    }
                    __syncthreads();
                    lam = S.lam;
                }
            }
        }
        if (FEAT || LEARN) {
            const Choice c = learned_phase<FEAT>(S, idx, p, q, sp, th2, th4, r4, lam, feat, theta_out, la);
            if (FEAT) continue;
            lam = c.lam;
            L = c.L;
        }
        if (tid == 0) lam_out[idx] = lam;

        // ---- coefficients (Eq. chebychev_coeff_shifted), FP64, from the table
        // cos(pi m / 2L), m = 0..L (other m by symmetry), in the free Psi
        // buffers; kept in FP32 for the recurrence's epilogue
        {
            double *tab = coef_tab(S), *hs = tab + (L + 1);
            for (int e = tid; e <= L; e += kThreads) tab[e] = cospi((double)e / (2.0 * L));
            if (tid == 0) S.s2 = (float)(2.0 / lam);
            __syncthreads();
            for (int l = tid; l < L; l += kThreads) hs[l] = response(sp, 0.5 * lam * (cos_from_tab(tab, 2 * l + 1, L) + 1.0));
            __syncthreads();
            for (int k = tid; k < L; k += kThreads) {
                // table index k (2l + 1) mod 4L, advanced by 2k per node
                const int M4 = 4 * L;
                int ix = k % M4;
                const int step = (2 * k) % M4;
                double a = 0.0;
                for (int l = 0; l < L; ++l) {
                    int mm = ix > 2 * L ? M4 - ix : ix;
                    a += (mm > L ? -tab[2 * L - mm] : tab[mm]) * hs[l];
                    ix += step;
                    if (ix >= M4) ix -= M4;
                }
                S.coef[k] = (float)(2.0 / (double)L * a);
            }
            __syncthreads();
        }

        // ---- shift: At = (2/lambda) G (operand), Psi_1 = At - Id, H = c0/2 Id + c1 Psi_1
        const float s2 = S.s2;
        const float c0h = 0.5f * S.coef[0], c1 = L > 1 ? S.coef[1] : 0.f;
        Frag z1, z0, h;   // Psi_{k-1}, Psi_{k-2}, H in the accumulator layout
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = frag_row(w, lane, e), c = frag_col(nt, lane, e);
                const bool in = r < p && c < p;
                const float at = in ? s2 * S.g[r * (kP + 1) + c] : 0.f;
                const float eye = (r == c && in) ? 1.f : 0.f;
                z1.v[nt][e] = at - eye;
                z0.v[nt][e] = eye;   // Psi_0 = Id
                h.v[nt][e] = c0h * eye + c1 * z1.v[nt][e];
                if (TC) {
                    put_hilo(S.ahi, S.alo, r * kLdB + c, at);
                } else {
                    reinterpret_cast<float *>(S.ahi)[r * kLdB + c] = at;
                }
            }
        if (TC) {
            frag_store_hilo(z1, S.zhi[1], S.zlo[1], kLdB, w, lane);
        } else {
            float *zf = zbuf_f32(S, 1);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) zf[frag_row(w, lane, e) * kLdB + frag_col(nt, lane, e)] = z1.v[nt][e];
        }
        __syncthreads();

        // ---- recurrence
        for (int k = 2; k < L; ++k) {
            const int bcur = (k - 1) & 1;   // buffer holding Psi_{k-1}
            frag_zero(acc);
            if (TC) {
                mma_tile<false, true>(acc, S.ahi, S.alo, kLdB, S.zhi[bcur], S.zlo[bcur], kLdB, p16, true, w, lane);
            } else {
                const float *af = reinterpret_cast<const float *>(S.ahi);
                const float *zf = zbuf_f32(S, bcur);
                fma_tile(acc, [&](int i, int kk) { return af[i * kLdB + kk]; },
                         [&](int kk, int j) { return zf[kk * kLdB + j]; }, p, w, lane);
            }
            const float ck = S.coef[k];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float zk = fmaf(2.f, acc.v[nt][e], fmaf(-2.f, z1.v[nt][e], -z0.v[nt][e]));
                    z0.v[nt][e] = z1.v[nt][e];
                    z1.v[nt][e] = zk;
                    h.v[nt][e] = fmaf(ck, zk, h.v[nt][e]);
                }
            // Psi_k into the other buffer; one barrier per step
            if (TC) {
                frag_store_hilo(z1, S.zhi[bcur ^ 1], S.zlo[bcur ^ 1], kLdB, w, lane);
            } else {
                float *zf = zbuf_f32(S, bcur ^ 1);
#pragma unroll
                for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        zf[frag_row(w, lane, e) * kLdB + frag_col(nt, lane, e)] = z1.v[nt][e];
            }
            __syncthreads();
        }

        // ---- final product: Y = X H (tall) or H X (wide), H through shared memory
        if (TC) {
            frag_store_hilo(h, S.ahi, S.alo, kLdB, w, lane);   // At no longer needed
        } else {
            float *hf = reinterpret_cast<float *>(S.ahi);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) hf[frag_row(w, lane, e) * kLdB + frag_col(nt, lane, e)] = h.v[nt][e];
        }
        __syncthreads();
        // D = H Xp in column blocks of 64; D(r, c) is Y(c, r) (m >= n) or Y(r, c)
        for (int b = 0; b < (q + 63) / 64; ++b) {
            frag_zero(acc);
            if (TC) {
                mma_tile<false, true>(acc, S.ahi, S.alo, kLdB, S.xhi + 64 * b, S.xlo + 64 * b, kLdX, p16, true, w,
                                      lane);
            } else {
                const float *xf = reinterpret_cast<const float *>(S.xhi);
                const float *hf = reinterpret_cast<const float *>(S.ahi);
                fma_tile(acc, [&](int i, int kk) { return hf[i * kLdB + kk]; },
                         [&](int kk, int j) { return xf[kk * kLdX + 64 * b + j]; }, p, w, lane);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = frag_row(w, lane, e), c = 64 * b + frag_col(nt, lane, e);
                    if (r < p && c < q) {
                        if (tall)
                            Yg[(int64_t)c * ldym + r] = acc.v[nt][e];
                        else
                            Yg[(int64_t)r * ldym + c] = acc.v[nt][e];
                    }
                }
        }
        __syncthreads();   // shared memory is reused by the next matrix
    }
}

}  // namespace
}  // namespace cpa

using namespace cpa;

struct cpa_batch_ctx {
    int device = 0;
    int count = 0;
    int num_sms = 0;
    BatchDesc *d_desc = nullptr;
    int *d_order = nullptr;
    double *d_lambda = nullptr;
    ShrinkParams *d_shrink = nullptr;
    int shrink_cap = 0;
    int *d_status = nullptr;
    int max_L = 0;
    int64_t total = 0;   // elements covered by the packed buffers
    std::vector<ShrinkParams> uploaded;   // shrink parameters currently on the device
    // learned serving (allocated on first use): L chosen per matrix, fallbacks
    int *d_L = nullptr, *d_nfb = nullptr;
    // launch configuration (cpa_batch_set_config / cpa_batch_tune): kernel
    // variant (CPA_BATCH_MMA_SYNC or CPA_BATCH_TCGEN05), CTAs per SM (0: the
    // occupancy limit), work order (CPA_ORDER_SIZE or CPA_ORDER_GIVEN)
    int variant = CPA_BATCH_MMA_SYNC, per_sm = 0, order_kind = CPA_ORDER_SIZE;
    int *d_order_given = nullptr;
};

namespace {
thread_local char g_berr[256] = "";
cpa_status bfail(cudaError_t e, const char *where) {
    snprintf(g_berr, sizeof g_berr, "%s: %s", where, cudaGetErrorString(e));
    return CPA_ERR_CUDA;
}
#define BCK(call)                                        \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return bfail(e_, #call);  \
    } while (0)
}  // namespace

extern "C" {

cpa_status cpa_batch_create(cpa_handle h, int count, const int64_t *off, const int32_t *m, const int32_t *n,
                            const int32_t *L, int L0, cpa_batch *out) {
    if (!h || !out || count < 1 || !off || !m || !n) return CPA_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<BatchDesc> desc(count);
    int max_L = 0;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const int mi = m[i], ni = n[i], Li = L ? L[i] : L0;
        if (mi < 1 || ni < 1 || std::min(mi, ni) > kP || std::max(mi, ni) > kQ || off[i] < 0 || Li < 1 ||
            Li > kMaxBatchTerms)
            return CPA_ERR_INVALID_ARG;
        desc[i] = BatchDesc{off[i], mi, ni, Li, 0, nullptr, nullptr, 0, 0};
        max_L = std::max(max_L, Li);
        total = std::max(total, off[i] + (int64_t)mi * ni);
    }
    // largest work first: (L - 2) p^3 + p^2 q
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    auto work = [&](int i) {
        const double p = std::min(desc[i].m, desc[i].n), q = std::max(desc[i].m, desc[i].n);
        return (desc[i].L - 2) * p * p * p + 2.0 * p * p * q;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });

    int device = 0;
    BCK(cudaGetDevice(&device));
    cpa_batch b = new cpa_batch_ctx();
    b->device = device;
    b->count = count;
    b->max_L = max_L;
    b->total = total;
    BCK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device));
    cudaError_t e = cudaMalloc(&b->d_desc, sizeof(BatchDesc) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_lambda, sizeof(double) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, 2 * sizeof(int));   // status, work counter
    if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order_given, sizeof(int) * count);
    if (e == cudaSuccess) {
        std::vector<int> ident(count);
        std::iota(ident.begin(), ident.end(), 0);
        e = cudaMemcpy(b->d_order_given, ident.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cpa_batch_destroy(b);
        return bfail(e, "cpa_batch_create");
    }
    *out = b;
    return CPA_OK;
}

cpa_status cpa_batch_destroy(cpa_batch b) {
    if (!b) return CPA_ERR_INVALID_ARG;
    cudaFree(b->d_desc);
    cudaFree(b->d_order);
    cudaFree(b->d_lambda);
    cudaFree(b->d_shrink);
    cudaFree(b->d_status);
    cudaFree(b->d_L);
    cudaFree(b->d_nfb);
    cudaFree(b->d_order_given);
    delete b;
    return CPA_OK;
}

const double *cpa_batch_lambdas(cpa_batch b) { return b ? b->d_lambda : nullptr; }

cpa_status cpa_batch_read_lambdas(cpa_batch b, double *host_out, void *stream) {
    if (!b || !host_out) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    int status = 0;
    BCK(cudaMemcpyAsync(host_out, b->d_lambda, sizeof(double) * b->count, cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    return status ? (cpa_status)status : CPA_OK;
}

}  // extern "C"

namespace {

// Validates and uploads the shrink parameters (only when they changed since
// the last upload of this plan; such a call synchronises the stream).
cpa_status upload_shrink(cpa_batch b, const cpa_shrink *s, int s_count, cudaStream_t st) {
    std::vector<ShrinkParams> sp(s_count);
    memset(sp.data(), 0, sizeof(ShrinkParams) * s_count);   // padding too: compared with memcmp
    for (int i = 0; i < s_count; ++i) {
        const cpa_shrink &x = s[i];
        bool ok = (x.kind == CPA_HARD || x.kind == CPA_SOFT) ? (x.tau >= 0.0 && std::isfinite(x.tau))
                  : (x.kind == CPA_WSOFT) ? (x.c >= 0.0 && x.eps > 0.0 && x.noise >= 0.0 && std::isfinite(x.c) &&
                                             std::isfinite(x.noise))
                                          : false;
        if (!ok) return CPA_ERR_INVALID_ARG;
        sp[i].kind = x.kind;
        sp[i].tau = x.tau;
        sp[i].c = x.c;
        sp[i].eps = x.eps;
        sp[i].noise = x.noise;
    }
    const bool same = b->uploaded.size() == sp.size() &&
                      memcmp(b->uploaded.data(), sp.data(), sizeof(ShrinkParams) * sp.size()) == 0;
    if (!same) {
        BCK(cudaStreamSynchronize(st));
        if (b->shrink_cap < s_count) {
            if (b->d_shrink) cudaFree(b->d_shrink);
            b->d_shrink = nullptr;
            BCK(cudaMalloc(&b->d_shrink, sizeof(ShrinkParams) * s_count));
            b->shrink_cap = s_count;
        }
        BCK(cudaMemcpy(b->d_shrink, sp.data(), sizeof(ShrinkParams) * s_count, cudaMemcpyHostToDevice));
        b->uploaded = sp;
    }
    return CPA_OK;
}

// Device buffers of one batched launch.
struct BatchRun {
    const BatchDesc *desc;
    const int *order;
    int count;
    const ShrinkParams *shrink;
    double *lambda_out;
    int *status;
    int num_sms;
    int variant;    // CPA_BATCH_MMA_SYNC or CPA_BATCH_TCGEN05 (tensor-core precisions)
    int per_sm;     // CTAs per SM of the mma.sync kernel, 0: its occupancy limit
};

template <bool TC, bool FEAT, bool LEARN>
cpa_status launch_run(const BatchRun &b, const float *dX, float *dY, int s_count, const double *lambda, int iters,
                      const int *L_override, float *feat, double *theta, const LearnArgs &la, cudaStream_t st) {
    if (TC && !FEAT && b.variant == CPA_BATCH_TCGEN05) {
        // tensor-core products (tcgen05, state in tensor memory)
        BCK(launch_batched_tc(b.desc, b.order, b.count, dX, dY, b.shrink, s_count > 1 ? 1 : 0, lambda, b.lambda_out,
                              iters, b.status, L_override, la, LEARN, b.num_sms, st));
        return CPA_OK;
    }
    const size_t smem = sizeof(BatchSmem);
    auto kern = batched_kernel<TC, FEAT, LEARN>;
    BCK(ensure_smem_limit((const void *)kern, (int)smem));
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    if (b.per_sm > 0 && b.per_sm < per_sm) per_sm = b.per_sm;
    const int grid = std::min(b.count, b.num_sms * per_sm);
    kern<<<grid, kThreads, smem, st>>>(b.desc, b.order, b.count, dX, dY, b.shrink, s_count > 1 ? 1 : 0, lambda,
                                       b.lambda_out, iters, b.status, L_override, feat, theta, la);
    BCK(cudaGetLastError());
    return CPA_OK;
}

template <bool TC, bool FEAT, bool LEARN>
cpa_status launch_batched(cpa_batch b, const float *dX, float *dY, int s_count, const double *lambda, int iters,
                          const int *L_override, float *feat, double *theta, const LearnArgs &la, cudaStream_t st) {
    const BatchRun r{b->d_desc, b->order_kind == CPA_ORDER_GIVEN ? b->d_order_given : b->d_order, b->count,
                     b->d_shrink, b->d_lambda, b->d_status, b->num_sms, b->variant, b->per_sm};
    return launch_run<TC, FEAT, LEARN>(r, dX, dY, s_count, lambda, iters, L_override, feat, theta, la, st);
}

cpa_status check_io(cpa_batch b, const float *dX, const float *dY) {
    const uintptr_t x0 = (uintptr_t)dX, y0 = (uintptr_t)dY, bytes = (uintptr_t)b->total * sizeof(float);
    if (dY && x0 < y0 + bytes && y0 < x0 + bytes) return CPA_ERR_INVALID_ARG;   // output overlaps input
    return CPA_OK;
}

cpa_status run_batched(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                       const double *lambda, int iters, int prec, float *dY, void *stream) {
    if (!h || !b || !dX || !dY || !s || (s_count != 1 && s_count != b->count) || iters < 0 || iters > 10000)
        return CPA_ERR_INVALID_ARG;
    if (prec != CPA_FP32 && prec != CPA_BF16 && prec != CPA_BF16X3) return CPA_ERR_UNSUPPORTED;
    cpa_status r = check_io(b, dX, dY);
    if (r != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    if ((r = upload_shrink(b, s, s_count, st)) != CPA_OK) return r;
    BCK(cudaMemsetAsync(b->d_status, 0, 2 * sizeof(int), st));
    const LearnArgs none{};
    if (prec != CPA_FP32)
        return launch_batched<true, false, false>(b, dX, dY, s_count, lambda, iters, nullptr, nullptr, nullptr, none,
                                                  st);
    return launch_batched<false, false, false>(b, dX, dY, s_count, lambda, iters, nullptr, nullptr, nullptr, none,
                                               st);
}

cpa_status ensure_learned_buffers(cpa_batch b) {
    if (b->d_L) return CPA_OK;
    if (cudaMalloc(&b->d_L, sizeof(int) * (size_t)b->count) != cudaSuccess ||
        cudaMalloc(&b->d_nfb, sizeof(int)) != cudaSuccess)
        return CPA_ERR_NO_MEMORY;
    return CPA_OK;
}

}  // namespace

extern "C" {

cpa_status cpa_svt_batched_plan(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                           const double *lambda, int iters, int prec, float *dY, void *stream) {
    return run_batched(h, b, dX, s, s_count, lambda, iters, prec, dY, stream);
}

cpa_status cpa_batch_features(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                              float *dF, double *dTheta, void *stream) {
    if (!h || !b || !dX || !s || !dF || !dTheta || (s_count != 1 && s_count != b->count)) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    cpa_status r = upload_shrink(b, s, s_count, st);
    if (r != CPA_OK) return r;
    BCK(cudaMemsetAsync(b->d_status, 0, 2 * sizeof(int), st));
    const LearnArgs none{};
    return launch_batched<true, true, false>(b, dX, nullptr, s_count, nullptr, 4, nullptr, dF, dTheta, none, st);
}

cpa_status cpa_svt_batched_learned(cpa_handle h, cpa_batch b, cpa_mlp net, const float *dX, const cpa_shrink *s,
                                   int s_count, double L_scale, int L_min, int L_max, int L_fallback, int use_lambda,
                                   double margin, int prec, float *dY, void *stream) {
    if (!h || !b || !net || !dX || !dY || !s || (s_count != 1 && s_count != b->count) || !(L_scale > 0.0) ||
        !(margin >= 0.0) || L_min < 1 || L_max < L_min || L_max > kMaxBatchTerms || L_fallback < 1 ||
        L_fallback > kMaxBatchTerms)
        return CPA_ERR_INVALID_ARG;
    if (prec != CPA_FP32 && prec != CPA_BF16 && prec != CPA_BF16X3) return CPA_ERR_UNSUPPORTED;
    int dims[4], net_device = -1;
    const float *P = mlp_device_params(net, dims, &net_device);
    if (!P || dims[0] != kFeatures || dims[1] != kHidden || dims[2] != kHidden || dims[3] != 2 ||
        net_device != b->device)
        return CPA_ERR_INVALID_ARG;   // the 12 -> 64 -> 64 -> 2 predictor, on the plan's device
    cpa_status r = check_io(b, dX, dY);
    if (r != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    if ((r = ensure_learned_buffers(b)) != CPA_OK) return r;
    if ((r = upload_shrink(b, s, s_count, st)) != CPA_OK) return r;
    BCK(cudaMemsetAsync(b->d_status, 0, 2 * sizeof(int), st));
    BCK(cudaMemsetAsync(b->d_nfb, 0, sizeof(int), st));
    LearnArgs la{P, L_scale, margin, L_min, L_max, L_fallback, use_lambda ? 1 : 0, b->d_L, b->d_nfb};
    if (prec != CPA_FP32)
        return launch_batched<true, false, true>(b, dX, dY, s_count, nullptr, kDefaultPowerIters, nullptr, nullptr,
                                                 nullptr, la, st);
    return launch_batched<false, false, true>(b, dX, dY, s_count, nullptr, kDefaultPowerIters, nullptr, nullptr,
                                              nullptr, la, st);
}

cpa_status cpa_batch_set_config(cpa_batch b, int variant, int ctas_per_sm, int order) {
    if (!b || (variant != CPA_BATCH_MMA_SYNC && variant != CPA_BATCH_TCGEN05) || ctas_per_sm < 0 ||
        ctas_per_sm > 2 || (order != CPA_ORDER_SIZE && order != CPA_ORDER_GIVEN))
        return CPA_ERR_INVALID_ARG;
    b->variant = variant;
    b->per_sm = ctas_per_sm;
    b->order_kind = order;
    return CPA_OK;
}

cpa_status cpa_batch_get_config(cpa_batch b, int *variant, int *ctas_per_sm, int *order) {
    if (!b) return CPA_ERR_INVALID_ARG;
    if (variant) *variant = b->variant;
    if (ctas_per_sm) *ctas_per_sm = b->per_sm;
    if (order) *order = b->order_kind;
    return CPA_OK;
}

cpa_status cpa_batch_tune(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count, int prec,
                          float *dY, int reps, int *chosen, double *ms, void *stream) {
    if (!h || !b || !chosen || reps < 1 || reps > 1000) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    const int saved[3] = {b->variant, b->per_sm, b->order_kind};
    double best = -1.0;
    int bc[3] = {saved[0], saved[1], saved[2]};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    cpa_status r = CPA_OK;
    int slot = 0;
    for (int variant = 0; variant < 2 && r == CPA_OK; ++variant)
        for (int per_sm = 1; per_sm <= 2 && r == CPA_OK; ++per_sm)
            for (int order = 0; order < 2 && r == CPA_OK; ++order, ++slot) {
                const bool run = !(variant == CPA_BATCH_TCGEN05 && (prec == CPA_FP32 || per_sm != 1));
                if (ms) ms[slot] = -1.0;
                if (!run) continue;
                b->variant = variant;
                b->per_sm = per_sm;
                b->order_kind = order;
                if ((r = cpa_svt_batched_plan(h, b, dX, s, s_count, nullptr, kDefaultPowerIters, prec, dY, stream)) !=
                    CPA_OK)
                    break;
                if (cudaEventRecord(e0, st) != cudaSuccess) { r = CPA_ERR_CUDA; break; }
                for (int k = 0; k < reps && r == CPA_OK; ++k)
                    r = cpa_svt_batched_plan(h, b, dX, s, s_count, nullptr, kDefaultPowerIters, prec, dY, stream);
                float t = 0.f;
                if (r != CPA_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                    if (r == CPA_OK) r = CPA_ERR_CUDA;
                    break;
                }
                const double mean = (double)t / reps;
                if (ms) ms[slot] = mean;
                if (best < 0.0 || mean < best) {
                    best = mean;
                    bc[0] = variant;
                    bc[1] = per_sm;
                    bc[2] = order;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = r == CPA_OK ? bc[0] : saved[0];
    b->per_sm = r == CPA_OK ? bc[1] : saved[1];
    b->order_kind = r == CPA_OK ? bc[2] : saved[2];
    chosen[0] = b->variant;
    chosen[1] = b->per_sm;
    chosen[2] = b->order_kind;
    return r;
}

cpa_status cpa_batch_read_choices(cpa_batch b, int *host_L, int *host_fallbacks, void *stream) {
    if (!b || !b->d_L) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    if (host_L) BCK(cudaMemcpyAsync(host_L, b->d_L, sizeof(int) * b->count, cudaMemcpyDeviceToHost, st));
    if (host_fallbacks) BCK(cudaMemcpyAsync(host_fallbacks, b->d_nfb, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    return CPA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Pointer form: a batch given as per-matrix device pointers, shapes, leading
// dimensions and orders (the patch-sized members of cpa_svt_batched and
// cpa_serve_learned).  The handle owns one PtrPlan: device descriptor
// buffers grown on demand and pinned host staging, uploaded on the call's
// stream; an event orders the reuse of the staging across calls.

namespace cpa {

struct PtrPlan {
    int device = 0, num_sms = 0, cap = 0;
    BatchDesc *d_desc = nullptr, *h_desc = nullptr;
    int *d_order = nullptr, *h_order = nullptr;
    ShrinkParams *d_shrink = nullptr, *h_shrink = nullptr;
    double *d_lam_in = nullptr, *h_lam = nullptr, *d_lam_out = nullptr;
    int *d_status = nullptr, *d_L = nullptr, *d_nfb = nullptr;
    cudaEvent_t staged = nullptr;
};

namespace {
void ptr_plan_free(PtrPlan *pp) {
    cudaFree(pp->d_desc);
    cudaFree(pp->d_order);
    cudaFree(pp->d_shrink);
    cudaFree(pp->d_lam_in);
    cudaFree(pp->d_lam_out);
    cudaFree(pp->d_status);
    cudaFree(pp->d_L);
    cudaFree(pp->d_nfb);
    cudaFreeHost(pp->h_desc);
    cudaFreeHost(pp->h_order);
    cudaFreeHost(pp->h_shrink);
    cudaFreeHost(pp->h_lam);
    pp->d_desc = pp->h_desc = nullptr;
    pp->d_order = pp->h_order = nullptr;
    pp->d_shrink = pp->h_shrink = nullptr;
    pp->d_lam_in = pp->h_lam = pp->d_lam_out = nullptr;
    pp->d_status = pp->d_L = pp->d_nfb = nullptr;
    pp->cap = 0;
}

cpa_status ptr_plan_reserve(PtrPlan *pp, int count, cudaStream_t st) {
    if (count <= pp->cap) return CPA_OK;
    BCK(cudaStreamSynchronize(st));
    if (pp->staged) BCK(cudaEventSynchronize(pp->staged));
    ptr_plan_free(pp);
    const int c = std::max(count, 256);
    cudaError_t e = cudaMalloc(&pp->d_desc, sizeof(BatchDesc) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_order, sizeof(int) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_shrink, sizeof(ShrinkParams) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_lam_in, sizeof(double) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_lam_out, sizeof(double) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_status, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_L, sizeof(int) * c);
    if (e == cudaSuccess) e = cudaMalloc(&pp->d_nfb, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&pp->h_desc, sizeof(BatchDesc) * c);
    if (e == cudaSuccess) e = cudaMallocHost(&pp->h_order, sizeof(int) * c);
    if (e == cudaSuccess) e = cudaMallocHost(&pp->h_shrink, sizeof(ShrinkParams) * c);
    if (e == cudaSuccess) e = cudaMallocHost(&pp->h_lam, sizeof(double) * c);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr_plan_free(pp);
        return CPA_ERR_NO_MEMORY;
    }
    pp->cap = c;
    return CPA_OK;
}
}  // namespace

PtrPlan *ptr_plan_create(int device, int num_sms) {
    PtrPlan *pp = new PtrPlan();
    pp->device = device;
    pp->num_sms = num_sms;
    return pp;
}

void ptr_plan_destroy(PtrPlan *pp) {
    if (!pp) return;
    if (pp->staged) {
        cudaEventSynchronize(pp->staged);
        cudaEventDestroy(pp->staged);
    }
    ptr_plan_free(pp);
    delete pp;
}

cpa_status ptr_plan_run(PtrPlan *pp, int count, const PtrItem *items, const double *lambda_host, int prec,
                        const float *net, const cpa_learn_rule *rule, cudaStream_t st, int variant) {
    if (count <= 0) return CPA_OK;
    cpa_status r = ptr_plan_reserve(pp, count, st);
    if (r != CPA_OK) return r;
    if (!pp->staged) BCK(cudaEventCreateWithFlags(&pp->staged, cudaEventDisableTiming));
    BCK(cudaEventSynchronize(pp->staged));   // the previous call's upload has read the staging
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        const PtrItem &it = items[i];
        pp->h_desc[i] = BatchDesc{0, it.m, it.n, it.L, 0, it.x, it.y, it.ldx, it.ldy};
        pp->h_shrink[i] = it.shrink;
        pp->h_order[i] = i;
        const double p = std::min(it.m, it.n), q = std::max(it.m, it.n);
        work[i] = (it.L - 2) * p * p * p + 2.0 * p * p * q;
        if (lambda_host) pp->h_lam[i] = lambda_host[i];
    }
    std::stable_sort(pp->h_order, pp->h_order + count, [&](int a, int b) { return work[a] > work[b]; });
    BCK(cudaMemcpyAsync(pp->d_desc, pp->h_desc, sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(pp->d_order, pp->h_order, sizeof(int) * count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(pp->d_shrink, pp->h_shrink, sizeof(ShrinkParams) * count, cudaMemcpyHostToDevice, st));
    if (lambda_host)
        BCK(cudaMemcpyAsync(pp->d_lam_in, pp->h_lam, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    BCK(cudaEventRecord(pp->staged, st));
    BCK(cudaMemsetAsync(pp->d_status, 0, 2 * sizeof(int), st));
    const BatchRun run{pp->d_desc, pp->d_order, count, pp->d_shrink, pp->d_lam_out, pp->d_status, pp->num_sms,
                       variant, 0};
    const bool tc = prec != CPA_FP32;
    if (net) {
        BCK(cudaMemsetAsync(pp->d_nfb, 0, sizeof(int), st));
        LearnArgs la{net, rule->L_scale, rule->margin, rule->L_min, std::min(rule->L_max, kMaxBatchTerms),
                     std::min(rule->L_fallback, kMaxBatchTerms), rule->use_lambda ? 1 : 0, pp->d_L, pp->d_nfb};
        if (tc)
            return launch_run<true, false, true>(run, nullptr, nullptr, count, nullptr, kDefaultPowerIters, nullptr,
                                                 nullptr, nullptr, la, st);
        return launch_run<false, false, true>(run, nullptr, nullptr, count, nullptr, kDefaultPowerIters, nullptr,
                                              nullptr, nullptr, la, st);
    }
    const LearnArgs none{};
    const double *lam = lambda_host ? pp->d_lam_in : nullptr;
    if (tc)
        return launch_run<true, false, false>(run, nullptr, nullptr, count, lam, kDefaultPowerIters, nullptr, nullptr,
                                              nullptr, none, st);
    return launch_run<false, false, false>(run, nullptr, nullptr, count, lam, kDefaultPowerIters, nullptr, nullptr,
                                           nullptr, none, st);
}

// Device arrays of the last run: the bound and (learned runs) the order of
// each member, in the order of the items passed; the fallback count.
const double *ptr_plan_lambdas(const PtrPlan *pp) { return pp->d_lam_out; }
const int *ptr_plan_orders(const PtrPlan *pp) { return pp->d_L; }
const int *ptr_plan_fallbacks(const PtrPlan *pp) { return pp->d_nfb; }
const int *ptr_plan_status(const PtrPlan *pp) { return pp->d_status; }

int batched_max_terms() { return kMaxBatchTerms; }

}  // namespace cpa
