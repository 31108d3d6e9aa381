// Batched CPA shrinkage on the tensor cores: one CTA of 512 threads per
// member matrix at a time (persistent over a size-sorted work list), for
// members with p = min(m, n) <= 128 and q = max(m, n) <= 4096 (X staged
// through shared memory in chunks of 256 columns for the Gram matrix and
// 256 output columns for the final product).
//
// Tensor-memory lane r holds row r of every p x p matrix of the member.
// Thread t = 128 cq + r (cq = 0..3) works on row r, columns [32 cq, 32 cq
// + 32) of the element-wise passes (a warp may only touch its own quarter
// of the lanes: warp w's lanes are 32 (w mod 4) .. + 31, which is row r's
// quarter); the scalar phases (power iteration, features, network) run on
// the threads of cq = 0, one per row.  Tensor-memory columns:
//   TMEM columns [0, 128)    product accumulator (the Gram matrix, A Psi_{k-1};
//                            the final product uses [0, 256))
//   [128, 256), [256, 384)   the ring Psi_{k-1}, Psi_{k-2} (FP32)
//   [384, 512)               the running sum H (FP32)
// Products are tcgen05.mma kind::f16 with M = 128 and N = round_up(p, 16)
// (the final product N = round_up(q, 16)), FP32 accumulate, the BF16 hi/lo
// split hi*hi + hi*lo + lo*hi, operands in shared memory as 128-byte
// swizzled K-major tiles written by the threads themselves (each thread
// writes its own row): X (Gram), At = (2/lambda) G and Psi_{k-1}
// (recurrence), H and X (final product).  The epilogue of a recurrence step
// reads the accumulator and the state from tensor memory, forms
//   Psi_k = 2 At Psi_{k-1} - 2 Psi_{k-1} - Psi_{k-2},  H += c_k Psi_k
// in FP32, writes Psi_k back in place of Psi_{k-2} and its BF16 parts into
// the operand tile of the next product (padding rows and columns beyond p
// are zero in every operand and state, so they stay zero).  The products read the operand's
// rows, A B^T, so G and every Psi_k are kept exactly symmetric (each takes
// its upper triangle's values, exchanged through shared memory), as the
// single-matrix tensor-core path does by mirroring upper tiles.  Lambda_max
// (power iteration, FP32
// with the FP64 final step), the coefficients (FP64 sums) and the learned
// choice follow the definitions of the CUDA-core batched kernel.
#include <algorithm>

#include "internal.h"
#include "tc_ptx.h"

namespace cpa {
namespace {

using namespace tc;

constexpr int kT = 512;                 // threads (16 warps): 4 column quarters x 128 rows
constexpr int kRows = 128;              // rows of a tile = tensor-memory lanes
constexpr int kP = kTcBatchP;           // rows of a member's p x p matrices
constexpr int kLdG = kP + 1;            // FP32 Gram matrix row stride (conflict-free rows)
constexpr int kChunkQ = 256;            // columns of X_p staged per Gram chunk / rows of X_p^T per output chunk
constexpr int kTcMaxTerms = 1024;
constexpr int kFeat = 12, kHid = 64;
constexpr uint64_t kEdgeXor = 0x5EEDULL;

// Shared memory (bytes from the 1024-aligned base):
//   R1 [0, 133120)     Gram phase: X_p hi (4 K-slices x 128 rows x 128 B) and lo;
//                      then the FP32 Gram matrix [128][129] at 0 and the
//                      Psi operand (2 slices, 128 rows) hi at 66560, lo at
//                      99328; final phase: X_p^T hi (2 slices x 256 rows) at
//                      0, lo at 65536
//   R2 [133120, +65536) At hi (2 slices x 128 rows) and lo; the FP64
//                      coefficient table before the shift; H hi/lo for the
//                      final product
//   small               coefficients, vectors, reductions, barrier
constexpr int kR1 = 133120, kR2 = 65536;
constexpr int kSlice128 = 128 * 128;            // one K slice of a 128-row tile
constexpr int kSlice256 = 256 * 128;
constexpr int kPsiHi = 66560, kPsiLo = kPsiHi + 2 * kSlice128;
constexpr int kXtLo = 2 * kSlice256;
constexpr int kXLo = 4 * kSlice128;

struct Small {
    float coef[kTcMaxTerms];      // c_k in FP32 (before: the predictor's scratch)
    float v[2][kP];             // power-iteration vectors
    float red[8];               // block-sum partials (warps 0-3), two sets of four
    double scal[4];             // lambda, chosen L (as double), spare
    double lam;
    float s2;
    int next_it;
    uint32_t tmem_slot;
    int abort_flag;
    alignas(8) uint64_t bar;
};
constexpr int kSmemBytes = kR1 + kR2 + (int)sizeof(Small) + 1024;

__device__ __forceinline__ uint32_t bf16bits(float v) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Eight consecutive values of row `row`, columns col0 .. col0 + 7 (col0 a
// multiple of 8), as BF16 hi and lo parts into 128-byte swizzled K-major
// tiles (K slice col0 / 64, 16-byte chunk (col0 % 64) / 8 XOR row % 8).
__device__ __forceinline__ void put8(uint8_t *hi, uint8_t *lo, int slice_bytes, int row, int col0, const float *v) {
    const int s = col0 >> 6, c = (col0 & 63) >> 3;
    const int off = s * slice_bytes + row * 128 + ((c ^ (row & 7)) << 4);
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
        const float r0 = v[2 * e] - __bfloat162float(h0), r1 = v[2 * e + 1] - __bfloat162float(h1);
        h[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[e] = bf16bits(r0) | (bf16bits(r1) << 16);
    }
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One element (row, col) as BF16 hi and lo parts into the same layout.
__device__ __forceinline__ void put1(uint8_t *hi, uint8_t *lo, int slice_bytes, int row, int col, float v) {
    const int s = col >> 6, c = (col & 63) >> 3;
    const int off = s * slice_bytes + row * 128 + ((c ^ (row & 7)) << 4) + (col & 7) * 2;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16 *>(lo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Zero `bytes` (a multiple of 16) of shared memory from p, all threads.
__device__ __forceinline__ void zero_smem(uint8_t *p, int bytes) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    for (int i = threadIdx.x; i < bytes / 16; i += kT) q[i] = make_uint4(0, 0, 0, 0);
}

// D[tmem d] (+)= sum over kslices K slices of A B^T with the BF16 split
// (hi*hi + hi*lo + lo*hi; accumulating onto D when acc0 = 1), then a commit
// to `bar`.  Issued by one thread.
__device__ __forceinline__ void issue_split_product(uint32_t d, const uint8_t *a_hi, const uint8_t *a_lo,
                                                    int a_slice, const uint8_t *b_hi, const uint8_t *b_lo, int b_slice,
                                                    int kslices, uint32_t idesc, uint64_t *bar, uint32_t acc0) {
    uint32_t acc = acc0;
#pragma unroll 1
    for (int seg = 0; seg < 3; ++seg) {
        const uint8_t *a = seg == 2 ? a_lo : a_hi;
        const uint8_t *b = seg == 1 ? b_lo : b_hi;
#pragma unroll 1
        for (int s = 0; s < kslices; ++s) {
            const uint64_t da = smem_desc(su32(a + s * a_slice)), db = smem_desc(su32(b + s * b_slice));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                mma_bf16(d, da + 2 * kk, db + 2 * kk, idesc, acc);
                acc = 1;
            }
        }
    }
    mma_commit(bar);
}

// Sixteen columns of this thread's lane at each of three addresses, one wait.
__device__ __forceinline__ void tmem_ld16x3(uint32_t ta, uint32_t tb, uint32_t tc, float *a, float *b, float *c) {
    uint32_t r[48];
#define CPA_LD16(base, addr)                                                                                         \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                                           \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"                                  \
                 : "=r"(r[base + 0]), "=r"(r[base + 1]), "=r"(r[base + 2]), "=r"(r[base + 3]), "=r"(r[base + 4]),   \
                   "=r"(r[base + 5]), "=r"(r[base + 6]), "=r"(r[base + 7]), "=r"(r[base + 8]), "=r"(r[base + 9]),   \
                   "=r"(r[base + 10]), "=r"(r[base + 11]), "=r"(r[base + 12]), "=r"(r[base + 13]),                 \
                   "=r"(r[base + 14]), "=r"(r[base + 15])                                                            \
                 : "r"(addr))
    CPA_LD16(0, ta);
    CPA_LD16(16, tb);
    CPA_LD16(32, tc);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        a[j] = __uint_as_float(r[j]);
        b[j] = __uint_as_float(r[16 + j]);
        c[j] = __uint_as_float(r[32 + j]);
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float *a) {
    uint32_t r[16];
    CPA_LD16(0, ta);
#undef CPA_LD16
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
    tmem_st8(taddr, v);
    tmem_st8(taddr + 8, v + 8);
}

// Block sum of one float per thread of the first 128 (the scalar phases'
// threads; the others pass 0 and only take part in the barrier); the
// partials alternate between two slot sets so one barrier per call suffices.
__device__ __forceinline__ float bsum(float x, float *red8, int &slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    float *r = red8 + 4 * (slot & 1);
    ++slot;
    if ((threadIdx.x & 31) == 0 && threadIdx.x < kRows) r[threadIdx.x >> 5] = x;
    __syncthreads();
    return (r[0] + r[1]) + (r[2] + r[3]);
}

__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float start_entry(uint64_t seed, int i) {
    return (float)((double)(splitmix(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// (G v)(row) from the FP32 Gram matrix, one thread per row; 0 for rows >= p.
__device__ __forceinline__ float gv_row(const float *g, int row, int p, const float *v) {
    float a0 = 0.f, a1 = 0.f;
    if (row < p) {
        const float *gr = g + row * kLdG;
        int j = 0;
        for (; j + 1 < p; j += 2) {
            a0 = fmaf(gr[j], v[j], a0);
            a1 = fmaf(gr[j + 1], v[j + 1], a1);
        }
        if (j < p) a0 = fmaf(gr[j], v[j], a0);
    }
    return a0 + a1;
}

}  // namespace
}  // namespace cpa

namespace cpa {
namespace {

struct TcChoice {
    double lam;
    int L;
};

// The learned choice for one member from the FP32 Gram matrix g (the
// definitions of cpa_batch_features and cpa_svt_batched_learned): the lower
// spectral edge, |G|_F^2 and the trace, the twelve features, the network in
// the summation order of its own forward kernel, the decision rule.
__device__ __noinline__ TcChoice tc_learned_phase(Small &S, const float *g, int idx, int p, int q, ShrinkParams sp,
                                                   float th2, float th4, float r4, double lam, const LearnArgs la) {
    const int tid = threadIdx.x;
    const bool own = tid < p;
    int rs = 0;
    __syncthreads();
    for (int i = tid; i < p; i += kT) S.v[0][i] = start_entry(kStartSeed ^ kEdgeXor, i);
    __syncthreads();
    float lmin = 0.f;
    int uc = 0;
    for (int t = 0; t <= 4; ++t) {
        const float a = gv_row(g, tid, p, S.v[uc]);
        const float ur = own ? S.v[uc][tid] : 0.f;
        if (t < 4) {
            const float nx = th4 * ur - a;
            const float n2 = bsum(own ? nx * nx : 0.f, S.red, rs);
            const float sc2 = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
            if (own) S.v[uc ^ 1][tid] = nx * sc2;
            __syncthreads();
            uc ^= 1;
        } else {
            const float num = bsum(ur * a, S.red, rs);
            const float den = bsum(ur * ur, S.red, rs);
            lmin = den > 0.f ? num / den : 0.f;
        }
    }
    float fro = 0.f;
    if (own)
        for (int c = 0; c < p; ++c) fro = fmaf(g[tid * kLdG + c], g[tid * kLdG + c], fro);
    fro = bsum(fro, S.red, rs);
    const float tr = bsum(own ? g[tid * kLdG + tid] : 0.f, S.red, rs);
    float *fv = S.coef;   // free until the coefficients are formed
    if (tid < kFeat) {
        const double tiny = 1e-30;
        const double E = tr > 0.f ? (double)tr : 1.0;
        const double t4 = fmax((double)th4, tiny * E);
        double thr2;
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
    __syncthreads();
    constexpr int oW1 = 0, ob1 = kHid * kFeat, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
                  ob3 = oW3 + 2 * kHid;
    float *h1 = fv + 16, *h2 = h1 + kHid, *yv = h2 + kHid;
    if (tid < kHid) {
        float a = __ldg(la.P + ob1 + tid);
        for (int j = 0; j < kFeat; ++j) a = fmaf(__ldg(la.P + oW1 + tid * kFeat + j), fv[j], a);
        h1[tid] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (tid < kHid) {
        float a = __ldg(la.P + ob2 + tid);
        for (int j = 0; j < kHid; ++j) a = fmaf(__ldg(la.P + oW2 + tid * kHid + j), h1[j], a);
        h2[tid] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (tid < 2) {
        float a = __ldg(la.P + ob3 + tid);
        for (int j = 0; j < kHid; ++j) a = fmaf(__ldg(la.P + oW3 + tid * kHid + j), h2[j], a);
        yv[tid] = a;
    }
    __syncthreads();
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
            if (ok_lam)
                lc = fmax(lp, floor_lam);
            else
                Lc = la.L_fallback;
        }
        la.L_out[idx] = Lc;
        if (!ok_L || !ok_lam) atomicAdd(la.nfallback, 1);
        S.scal[0] = lc;
        S.next_it = Lc;
    }
    __syncthreads();
    const TcChoice c{S.scal[0], S.next_it};
    __syncthreads();
    return c;
}

}  // namespace
}  // namespace cpa

namespace cpa {
namespace {

template <bool LEARN>
__global__ void __launch_bounds__(kT, 1)
    batched_tc_kernel(const BatchDesc *__restrict__ descs, const int *__restrict__ order, int count,
                      const float *__restrict__ X, float *__restrict__ Y, const ShrinkParams *__restrict__ shr,
                      int shr_stride, const double *__restrict__ lam_in, double *__restrict__ lam_out, int iters,
                      int *__restrict__ status, const int *__restrict__ L_in, const LearnArgs la) {
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *R1 = base, *R2 = base + kR1;
    Small &S = *reinterpret_cast<Small *>(base + kR1 + kR2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kRows - 1), c0q = 32 * (tid / kRows);   // this thread's row and 32-column chunk
    constexpr uint32_t cACC = 0, cPSI0 = 128, cPSI1 = 256, cH = 384;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&S.tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's 32 lanes (rows)
    volatile int *abort_flag = &S.abort_flag;
    uint32_t phase = 0;

    // One split product into TMEM columns [0, N): operands written by every
    // thread are made visible to the tensor core, one thread issues, all wait.
    auto run_product = [&](const uint8_t *ahi, const uint8_t *alo, int aslice, const uint8_t *bhi,
                           const uint8_t *blo, int bslice, int kslices, int N, uint32_t acc0 = 0) -> bool {
        tmem_st_wait();
        fence_proxy_async();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            issue_split_product(tmem + cACC, ahi, alo, aslice, bhi, blo, bslice, kslices, idesc_bf16(128, N), &S.bar,
                                acc0);
        }
        mbar_wait(&S.bar, phase, abort_flag);
        phase ^= 1;
        fence_after();
        __syncthreads();
        return *abort_flag == 0;
    };

    for (;;) {
        if (tid == 0) S.next_it = atomicAdd(status + 1, 1);
        __syncthreads();
        const int it = S.next_it;
        if (it >= count || *abort_flag) break;
        const int idx = order[it];
        const BatchDesc d = descs[idx];
        const int m = d.m, n = d.n;
        int L = L_in ? L_in[idx] : d.L;
        const bool tall = m >= n;
        const int p = tall ? n : m, q = tall ? m : n;
        const int Np = (p + 15) & ~15, Kp = (p + 63) & ~63;
        const float *Xg = d.x ? d.x : X + d.off;
        float *Yg = d.x ? d.y : Y + d.off;
        const int64_t ldxm = d.x ? d.ldx : n, ldym = d.x ? d.ldy : n;
        const ShrinkParams sp = shr[shr_stride ? idx : 0];
        const bool own = tid < p;        // scalar phases: thread tid < 128 is row tid
        const bool rowin = row < p;      // element-wise passes

        // ---- Gram G = X_p X_p^T, X_p = X^T when m >= n, else X (p x q):
        // K chunks of 256 columns of X_p staged in R1 (zero padded) and
        // accumulated in tensor memory
        bool ok = true;
        for (int k0 = 0; k0 < q && ok; k0 += kChunkQ) {
            const int kc = min(kChunkQ, q - k0);
            zero_smem(R1, 2 * kXLo);
            __syncthreads();
            if (tall) {   // X_p[r][k0 + c] = X[k0 + c][r]: rows of X are contiguous in r
                for (int e = tid; e < kc * p; e += kT) {
                    const int c = e / p, r = e - c * p;
                    put1(R1, R1 + kXLo, kSlice128, r, c, __ldg(Xg + (int64_t)(k0 + c) * ldxm + r));
                }
            } else {      // X_p[r][k0 + c] = X[r][k0 + c]
                for (int e = tid; e < p * kc; e += kT) {
                    const int r = e / kc, c = e - r * kc;
                    put1(R1, R1 + kXLo, kSlice128, r, c, __ldg(Xg + (int64_t)r * ldxm + k0 + c));
                }
            }
            ok = run_product(R1, R1 + kXLo, kSlice128, R1, R1 + kXLo, kSlice128, ((kc + 63) & ~63) / 64, Np,
                             k0 > 0 ? 1u : 0u);
        }
        if (!ok) break;
        float *g = reinterpret_cast<float *>(R1);
        if (c0q < Np) {
            float a[32];
            tmem_ld32(trow + cACC + c0q, a);
            if (rowin)
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (c0q + e < p) g[row * kLdG + c0q + e] = a[e];
        }
        __syncthreads();
        // exactly symmetric G: the lower triangle takes the upper one (the
        // products below multiply by the operand's rows, A B^T, which is
        // A B only for an exactly symmetric B; rounding asymmetry would grow
        // along the recurrence)
        if (rowin)
            for (int j = c0q; j < min(c0q + 32, row); ++j) g[row * kLdG + j] = g[j * kLdG + row];
        __syncthreads();

        // ---- Lambda_max: power iteration (definition of cpa_lambda_bound)
        double lam = lam_in ? lam_in[idx] : 0.0;
        float th2 = 0.f, th4 = 0.f, r4 = 0.f;
        int rs = 0;
        if (!(lam > 0.0) || LEARN) {
            const float x0 = own ? start_entry(kStartSeed, tid) : 0.f;
            if (own) S.v[0][tid] = x0;
            float nrm2 = bsum(x0 * x0, S.red, rs);
            int cur = 0;
            const int its = (LEARN && la.use_lambda) ? 4 : iters;
            for (int t = 0; t <= its; ++t) {
                const float sc = nrm2 > 0.f ? 1.f / sqrtf(nrm2) : 0.f;
                const float a = gv_row(g, tid, p, S.v[cur]) * sc;
                const float vt = own ? S.v[cur][tid] : 0.f;
                if (own) S.v[cur ^ 1][tid] = a;
                if (LEARN && t < its && t < 4) {
                    const float th = bsum(vt * a, S.red, rs) * sc;
                    if (t == 1) th2 = th;
                    if (t == 3) {
                        th4 = th;
                        const float dd = own ? a - th * vt * sc : 0.f;
                        r4 = sqrtf(fmaxf(bsum(dd * dd, S.red, rs), 0.f));
                    }
                }
                if (t < its) {
                    nrm2 = bsum(own ? a * a : 0.f, S.red, rs);
                    cur ^= 1;
                } else {
                    const float vu = vt * sc;
                    const float th = bsum(vu * a, S.red, rs);
                    const float dd = own ? a - th * vu : 0.f;
                    const float r2 = bsum(dd * dd, S.red, rs);
                    const float tr = bsum(own ? g[tid * kLdG + tid] : 0.f, S.red, rs);
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
        if (LEARN) {
            const TcChoice c = tc_learned_phase(S, g, idx, p, q, sp, th2, th4, r4, lam, la);
            lam = c.lam;
            L = c.L;
        }
        if (tid == 0) lam_out[idx] = lam;

        // ---- coefficients (Eq. chebychev_coeff_shifted), FP64 sums in R2,
        // kept in FP32
        {
            double *tab = reinterpret_cast<double *>(R2), *hs = tab + (L + 1);
            for (int e = tid; e <= L; e += kT) tab[e] = cospi((double)e / (2.0 * L));
            if (tid == 0) S.s2 = (float)(2.0 / lam);
            __syncthreads();
            for (int l = tid; l < L; l += kT) {
                int mm = (2 * l + 1) % (4 * L);
                if (mm > 2 * L) mm = 4 * L - mm;
                hs[l] = response(sp, 0.5 * lam * ((mm > L ? -tab[2 * L - mm] : tab[mm]) + 1.0));
            }
            __syncthreads();
            for (int k = tid; k < L; k += kT) {
                const int M4 = 4 * L;
                int ix = k % M4;
                const int step = (2 * k) % M4;
                double a = 0.0;
                for (int l = 0; l < L; ++l) {
                    const int mm = ix > 2 * L ? M4 - ix : ix;
                    a += (mm > L ? -tab[2 * L - mm] : tab[mm]) * hs[l];
                    ix += step;
                    if (ix >= M4) ix -= M4;
                }
                S.coef[k] = (float)(2.0 / (double)L * a);
            }
            __syncthreads();
        }

        // ---- shift: At = (2/lambda) G (operand in R2), Psi_1 = At - Id,
        // Psi_0 = Id, H = c_0/2 Id + c_1 Psi_1 (tensor memory), Psi_1's BF16
        // parts (operand in R1)
        {
            const float s2 = S.s2, c0h = 0.5f * S.coef[0], c1 = L > 1 ? S.coef[1] : 0.f;
            if (c0q < Kp) {
#pragma unroll
                for (int hf = 0; hf < 32; hf += 16) {
                    const int c0 = c0q + hf;
                    float at[16], z1[16], z0[16], hh[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = c0 + e;
                        const bool in = rowin && j < p;
                        const float eye = (in && j == row) ? 1.f : 0.f;
                        at[e] = in ? s2 * g[row * kLdG + j] : 0.f;
                        z1[e] = at[e] - eye;
                        z0[e] = eye;
                        hh[e] = fmaf(c1, z1[e], c0h * eye);
                    }
#pragma unroll
                    for (int u = 0; u < 16; u += 8) {
                        put8(R2, R2 + 2 * kSlice128, kSlice128, row, c0 + u, at + u);
                        put8(R1 + kPsiHi, R1 + kPsiLo, kSlice128, row, c0 + u, z1 + u);
                    }
                    tmem_st16(trow + cPSI1 + c0, z1);
                    tmem_st16(trow + cPSI0 + c0, z0);
                    tmem_st16(trow + cH + c0, hh);
                }
            }
        }

        // ---- recurrence Psi_k = 2 At Psi_{k-1} - 2 Psi_{k-1} - Psi_{k-2}, H += c_k Psi_k
        bool alive = true;
        for (int k = 2; k < L && alive; ++k) {
            alive = run_product(R2, R2 + 2 * kSlice128, kSlice128, R1 + kPsiHi, R1 + kPsiLo, kSlice128, Kp / 64, Np);
            if (!alive) break;
            const float ck = S.coef[k];
            const uint32_t sPrev = ((k - 1) & 1) ? cPSI1 : cPSI0, sOld = (k & 1) ? cPSI1 : cPSI0;
            // pass 1: row tid of 2 At Psi_{k-1} - 2 Psi_{k-1} - Psi_{k-2} into
            // the FP32 scratch (the Gram matrix's space, free after the shift)
            // (every row, including the zero padding rows, so that pass 2
            // reads written values only)
            float *w = reinterpret_cast<float *>(R1);
            if (c0q < Np) {
#pragma unroll
                for (int hf = 0; hf < 32; hf += 16) {
                    const int c0 = c0q + hf;
                    float a[16], z1[16], z0[16];
                    tmem_ld16x3(trow + cACC + c0, trow + sPrev + c0, trow + sOld + c0, a, z1, z0);
                    float *wr = w + row * kLdG + c0;
#pragma unroll
                    for (int e = 0; e < 16; ++e) wr[e] = fmaf(2.f, a[e], fmaf(-2.f, z1[e], -z0[e]));
                }
            }
            __syncthreads();
            // pass 2: Psi_k exactly symmetric (the upper triangle's values),
            // into the ring, the running sum and the next product's operand;
            // the entries of padding columns j >= p are the zeros pass 1
            // formed from zero operands and state, padding rows stay zero
            if (c0q < Np) {
#pragma unroll
                for (int hf = 0; hf < 32; hf += 16) {
                    const int c0 = c0q + hf;
                    float v[16], hh[16];
                    tmem_ld16(trow + cH + c0, hh);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = c0 + e;
                        const float *src = j >= row ? w + row * kLdG + j : w + j * kLdG + row;
                        v[e] = rowin ? *src : 0.f;
                        hh[e] = fmaf(ck, v[e], hh[e]);
                    }
                    tmem_st16(trow + sOld + c0, v);
                    tmem_st16(trow + cH + c0, hh);
                    put8(R1 + kPsiHi, R1 + kPsiLo, kSlice128, row, c0, v);
                    put8(R1 + kPsiHi, R1 + kPsiLo, kSlice128, row, c0 + 8, v + 8);
                }
            }
        }
        if (!alive) break;

        // ---- final product D = H X_p (p x q): H's BF16 parts (operand in
        // R2), X_p^T (q rows of p, operand in R1)
        tmem_st_wait();
        __syncthreads();
        if (c0q < Kp) {
            float hh[32];
            tmem_ld32(trow + cH + c0q, hh);
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if (!(rowin && c0q + e < p)) hh[e] = 0.f;
#pragma unroll
            for (int u = 0; u < 32; u += 8) put8(R2, R2 + 2 * kSlice128, kSlice128, row, c0q + u, hh + u);
        }
        // X_p^T (q rows of p) in chunks of 256 rows staged in R1; each
        // chunk's product D[:, n0 .. n0 + 256) goes straight to Y
        for (int n0 = 0; n0 < q && ok; n0 += kChunkQ) {
            const int nc = min(kChunkQ, q - n0), Nc = (nc + 15) & ~15;
            zero_smem(R1, 2 * kXtLo);
            __syncthreads();
            if (tall) {   // X_p^T[rr][k] = X[n0 + rr][k]
                for (int e = tid; e < nc * p; e += kT) {
                    const int rr = e / p, k = e - rr * p;
                    put1(R1, R1 + kXtLo, kSlice256, rr, k, __ldg(Xg + (int64_t)(n0 + rr) * ldxm + k));
                }
            } else {      // X_p^T[rr][k] = X[k][n0 + rr]
                for (int e = tid; e < p * nc; e += kT) {
                    const int k = e / nc, rr = e - k * nc;
                    put1(R1, R1 + kXtLo, kSlice256, rr, k, __ldg(Xg + (int64_t)k * ldxm + n0 + rr));
                }
            }
            ok = run_product(R2, R2 + 2 * kSlice128, kSlice128, R1, R1 + kXtLo, kSlice256, Kp / 64, Nc);
            if (!ok) break;
            for (int c0 = c0q; c0 < Nc; c0 += 4 * 32) {
                float dv[32];
                tmem_ld32(trow + cACC + c0, dv);
                if (rowin)
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const int jq = n0 + c0 + e;
                        if (c0 + e < nc) {
                            if (tall)
                                Yg[(int64_t)jq * ldym + row] = dv[e];
                            else
                                Yg[(int64_t)row * ldym + jq] = dv[e];
                        }
                    }
            }
        }
        if (!ok) break;
        tmem_st_wait();
        __syncthreads();   // shared and tensor memory are reused by the next member
    }

    if (tid == 0 && *abort_flag) atomicExch(status, (int)CPA_ERR_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

cudaError_t launch_batched_tc(const BatchDesc *desc, const int *order, int count, const float *X, float *Y,
                              const ShrinkParams *shr, int shr_stride, const double *lam_in, double *lam_out,
                              int iters, int *status, const int *L_in, const LearnArgs &la, bool learn,
                              int num_sms, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const void *fn = learn ? (const void *)batched_tc_kernel<true> : (const void *)batched_tc_kernel<false>;
    cudaError_t r = ensure_smem_limit(fn, kSmemBytes);
    if (r != cudaSuccess) return r;
    const int grid = std::min(count, num_sms);
    if (learn)
        batched_tc_kernel<true><<<grid, kT, kSmemBytes, st>>>(desc, order, count, X, Y, shr, shr_stride, lam_in,
                                                             lam_out, iters, status, L_in, la);
    else
        batched_tc_kernel<false><<<grid, kT, kSmemBytes, st>>>(desc, order, count, X, Y, shr, shr_stride, lam_in,
                                                              lam_out, iters, status, L_in, la);
    return cudaGetLastError();
}

}  // namespace cpa
