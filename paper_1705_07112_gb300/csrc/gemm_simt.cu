// FP32 CUDA-core GEMM with the fused CPA epilogue: the "plain FP32" path.
//
// Tile 128 x 128 x 16, 256 threads, 8 x 8 outputs per thread split as two
// 4-wide groups 64 apart (conflict-free float4 shared-memory reads), two
// shared-memory buffers with a register prefetch of the next K slice.
// Operands may be K-major or MN-major so that the Gram product X^T X, the
// recurrence A Psi and the final product X H all read X in place.
#include "internal.h"

namespace cpa {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

__device__ __forceinline__ void epi_store(const Epilogue &e, float ck, int i, int j, float acc) {
    float v = e.s_acc * acc;
    if (e.C) v = fmaf(e.s_c, e.C[(int64_t)i * e.ldc + j], v);
    if (e.C2) v = fmaf(e.s_c2, e.C2[(int64_t)i * e.ldc2 + j], v);
    if (i == j) v += epilogue_diag(e);
    e.D[(int64_t)i * e.ldd + j] = v;
    if (e.H) {
        float *hp = e.H + (int64_t)i * e.ldh + j;
        *hp = fmaf(ck, v, *hp);
    }
    if (e.Dhi) {
        __nv_bfloat16 hi = __float2bfloat16_rn(v);
        e.Dhi[(int64_t)i * e.ldb + j] = hi;
        if (e.Dlo) e.Dlo[(int64_t)i * e.ldb + j] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    if (e.symmetric_upper && i != j) {
        // mirror into the lower triangle (the tile (j,i) is not computed)
        e.D[(int64_t)j * e.ldd + i] = v;
        if (e.H) {
            float *hp = e.H + (int64_t)j * e.ldh + i;
            *hp = fmaf(ck, v, *hp);
        }
        if (e.Dhi) {
            __nv_bfloat16 hi = __float2bfloat16_rn(v);
            e.Dhi[(int64_t)j * e.ldb + i] = hi;
            if (e.Dlo) e.Dlo[(int64_t)j * e.ldb + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
    }
}

template <bool AK, bool BKM>
__global__ void __launch_bounds__(NT) gemm_f32_kernel(int M, int N, int K, const float *__restrict__ A,
                                                      int64_t lda, const float *__restrict__ B,
                                                      int64_t ldb, Epilogue e) {
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];

    int bm = blockIdx.y, bn = blockIdx.x;
    if (e.symmetric_upper && bn < bm) return;   // lower tiles mirrored by (bn, bm)
    const int m0 = bm * BM, n0 = bn * BN;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float ra[8], rb[8];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int idx = tid + r * NT;
            int i, k;
            if (AK) { k = idx % BK; i = idx / BK; } else { i = idx % BM; k = idx / BM; }
            int gi = m0 + i, gk = k0 + k;
            ra[r] = (gi < M && gk < K) ? (AK ? A[(int64_t)gi * lda + gk] : A[(int64_t)gk * lda + gi]) : 0.f;
            int j, kb;
            if (BKM) { kb = idx % BK; j = idx / BK; } else { j = idx % BN; kb = idx / BN; }
            int gj = n0 + j, gkb = k0 + kb;
            rb[r] = (gj < N && gkb < K) ? (BKM ? B[(int64_t)gj * ldb + gkb] : B[(int64_t)gkb * ldb + gj]) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int idx = tid + r * NT;
            int i, k;
            if (AK) { k = idx % BK; i = idx / BK; } else { i = idx % BM; k = idx / BM; }
            As[buf][k][i] = ra[r];
            int j, kb;
            if (BKM) { kb = idx % BK; j = idx / BK; } else { j = idx % BN; kb = idx / BN; }
            Bs[buf][kb][j] = rb[r];
        }
    };

    const int nk = (K + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        int cur = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], b[8];
            float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) store(cur ^ 1);
        __syncthreads();
    }

    const float ck = e.H ? (float)e.coef[e.k] : 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int gi = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int gj = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (gj >= N) continue;
            if (e.symmetric_upper && bm == bn && gj < gi) continue;   // diagonal tile: upper half only
            epi_store(e, ck, gi, gj, acc[i][j]);
        }
    }
}

}  // namespace

cudaError_t gemm_f32(int M, int N, int K, const float *A, int64_t lda, bool a_kmajor, const float *B,
                     int64_t ldb, bool b_kmajor, const Epilogue &e, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (a_kmajor && b_kmajor)
        gemm_f32_kernel<true, true><<<grid, NT, 0, st>>>(M, N, K, A, lda, B, ldb, e);
    else if (!a_kmajor && !b_kmajor)
        gemm_f32_kernel<false, false><<<grid, NT, 0, st>>>(M, N, K, A, lda, B, ldb, e);
    else if (a_kmajor && !b_kmajor)
        gemm_f32_kernel<true, false><<<grid, NT, 0, st>>>(M, N, K, A, lda, B, ldb, e);
    else
        gemm_f32_kernel<false, true><<<grid, NT, 0, st>>>(M, N, K, A, lda, B, ldb, e);
    return cudaGetLastError();
}

}  // namespace cpa
