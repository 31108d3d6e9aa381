// Completion ADMM of Section V, Comparison with Existing Methods: the inpainting problem of Section V, Texture Image Inpainting
// (Eq. texture_repaire4) without its average term, in the ADMM form of
// the appendix ADMM Applicable Forms, Texture Image Inpainting (Eq. admm_algorithm_inp, the z^(5) block dropped) around the CPA
// shrinkage.  z = K l with K = [Id; Psi; Omega; Id], Psi the orthonormal 2-D
// DCT (Psi l = C_m L C_n^T), Omega the observation mask:
//   l = (a1 + Psi^T a2 + omega a3 + a4) / (3 + omega),  a_i = z_i - u_i
//   z1 = prox_{(1/rho)|.|_*}(l + u1)        cpa_svt, soft, tau = 1/rho
//   z2 = prox_{(eta/rho)|.|_1}(Psi l + u2)   entrywise soft threshold
//   z3 = omega i                             the observed values
//   z4 = min(max(l + u4, 0), 1)
//   u += K l - z
// Start (Section V, Texture Image Inpainting): l = u = 1, z = K l.
//
// Device state (FP32, m x n, row stride n, owned by the solver): u1..u4,
// S = a1 + omega a3 + a4 (the spatial part of the next least-squares
// numerator), A2 = a2 (DCT domain), W = l + u1 (the next shrinkage input),
// Z1 (the shrinkage output) and two transform scratch arrays; l lives in the
// caller's output.  Per iteration: Q = Psi^T A2 (two products), the
// least-squares kernel (l, W and the sums of E_t), cpa_svt(W) -> Z1,
// P = Psi l (two products), the update kernel (z2..z4, u, A2, S).
// The products run in FP32 on the CUDA cores when prec is FP32, else on the
// tensor cores with BF16 hi/lo operands and three products each (hi hi +
// hi lo + lo hi, about 2^-16 relative error): C_m, C_n and their transposes
// are split once, the other operand and the intermediate once per pass, and
// each pass produces its intermediate transposed so that both products read
// K-major operands.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace cpa {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float soft_l1(float x, float t) {
    const float a = fabsf(x) - t;
    return a > 0.f ? copysignf(a, x) : 0.f;
}

// l = u = 1, S = omega (omega - 1) = 0; A2 = Psi 1 - 1 follows from P.
__global__ void init_kernel(int m, int n, float *l, int64_t ldl, float *u1, float *u2, float *u3, float *u4,
                            float *S) {
    const int64_t total = (int64_t)m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        l[i * ldl + j] = 1.f;
        u1[e] = 1.f;
        u2[e] = 1.f;
        u3[e] = 1.f;
        u4[e] = 1.f;
        S[e] = 0.f;
    }
}

__global__ void init_a2_kernel(int64_t total, const float *P, float *A2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        A2[e] = P[e] - 1.f;
}

// Least-squares step: l_new = (S + Q) / (3 + omega), W = l_new + u1;
// acc[0] += |l_new - l|^2, acc[1] += |l_new|^2.
__global__ void __launch_bounds__(kThreads)
    ls_kernel(int m, int n, const uint8_t *__restrict__ mask, int64_t ldm, const float *__restrict__ S,
              const float *__restrict__ Q, const float *__restrict__ u1, float *__restrict__ l, int64_t ldl,
              float *__restrict__ W, double *__restrict__ acc) {
    const int64_t total = (int64_t)m * n;
    double dsum = 0.0, lsum = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        const float om = mask[i * ldm + j] ? 1.f : 0.f;
        const float ln = (S[e] + Q[e]) / (3.f + om);
        const float lo = l[i * ldl + j];
        const double d = (double)ln - (double)lo;
        dsum += d * d;
        lsum += (double)ln * (double)ln;
        l[i * ldl + j] = ln;
        W[e] = ln + u1[e];
    }
    dsum = warp_sum(dsum);
    lsum = warp_sum(lsum);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, dsum);
        atomicAdd(acc + 1, lsum);
    }
}

// z and u updates from l, z1 = Z1 and P = Psi l; the next a2 and S.
__global__ void __launch_bounds__(kThreads)
    update_kernel(int m, int n, const float *__restrict__ I, int64_t ldi, const uint8_t *__restrict__ mask,
                  int64_t ldm, const float *__restrict__ l, int64_t ldl, const float *__restrict__ Z1,
                  const float *__restrict__ P, float *__restrict__ u1, float *__restrict__ u2,
                  float *__restrict__ u3, float *__restrict__ u4, float *__restrict__ A2, float *__restrict__ S,
                  float tau_l1) {
    const int64_t total = (int64_t)m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        const float om = mask[i * ldm + j] ? 1.f : 0.f;
        const float le = l[i * ldl + j];
        const float z1 = Z1[e], p = P[e];
        float a = u1[e], b = u2[e], c = u3[e], d = u4[e];
        const float z2 = soft_l1(p + b, tau_l1);
        const float z3 = om * I[i * ldi + j];
        const float z4 = fminf(fmaxf(le + d, 0.f), 1.f);
        a += le - z1;
        b += p - z2;
        c += om * le - z3;
        d += le - z4;
        u1[e] = a;
        u2[e] = b;
        u3[e] = c;
        u4[e] = d;
        A2[e] = z2 - b;
        S[e] = (z1 - a) + om * (z3 - c) + (z4 - d);
    }
}

}  // namespace
}  // namespace cpa

using namespace cpa;

struct cpa_completion_ctx {
    cpa_handle h = nullptr;
    int device = 0;
    int num_sms = 0;
    int64_t m = 0, n = 0;
    float *Cm = nullptr, *Cn = nullptr;   // orthonormal DCT-II, m x m and n x n (row stride m, n)
    float *state = nullptr;               // u1..u4, S, A2, W, Z1, T1, T2: 10 m n floats
    double *acc = nullptr;
    int acc_cap = 0;
    // tensor-core operands (BF16 hi/lo): C_m, C_m^T (row stride bm), C_n,
    // C_n^T (row stride bn), an m x n pass input (stride bn) and an n x m
    // intermediate (stride bm); bm, bn = m, n rounded up to 8
    int64_t bm = 0, bn = 0;
    __nv_bfloat16 *bf = nullptr;
    __nv_bfloat16 *Cmh = nullptr, *Cml = nullptr, *CmTh = nullptr, *CmTl = nullptr;
    __nv_bfloat16 *Cnh = nullptr, *Cnl = nullptr, *CnTh = nullptr, *CnTl = nullptr;
    __nv_bfloat16 *Xh = nullptr, *Xl = nullptr, *Th = nullptr, *Tl = nullptr;
};

namespace {
cpa_status ccuda(cudaError_t e) { return e == cudaSuccess ? CPA_OK : CPA_ERR_CUDA; }

// Tensor-core pass: out = C_m X C_n^T (forward) or C_m^T X C_n.  The
// intermediate Y^T (n x m, in tmp) = C_n X^T (forward) or C_n^T X^T.
cudaError_t dct2_tc(const cpa_completion_ctx *c, const float *X, int64_t ldx, bool transposed, float *tmp,
                    float *out, cudaStream_t st) {
    const int m = (int)c->m, n = (int)c->n;
    cudaError_t r;
    if ((r = split_bf16(X, m, n, ldx, false, c->Xh, c->Xl, c->bn, st)) != cudaSuccess) return r;
    TcOperand a1, b1, a2, b2;
    a1.hi = transposed ? c->CnTh : c->Cnh;
    a1.lo = transposed ? c->CnTl : c->Cnl;
    a1.ld = c->bn;
    a1.rows = n;
    b1.hi = c->Xh;
    b1.lo = c->Xl;
    b1.ld = c->bn;
    b1.rows = m;
    Epilogue e1;
    e1.D = tmp;
    e1.ldd = m;
    if ((r = gemm_tc(n, m, n, a1, b1, 3, e1, st, c->num_sms)) != cudaSuccess) return r;
    if ((r = split_bf16(tmp, n, m, m, false, c->Th, c->Tl, c->bm, st)) != cudaSuccess) return r;
    a2.hi = transposed ? c->CmTh : c->Cmh;
    a2.lo = transposed ? c->CmTl : c->Cml;
    a2.ld = c->bm;
    a2.rows = m;
    b2.hi = c->Th;
    b2.lo = c->Tl;
    b2.ld = c->bm;
    b2.rows = n;
    Epilogue e2;
    e2.D = out;
    e2.ldd = n;
    return gemm_tc(m, n, m, a2, b2, 3, e2, st, c->num_sms);
}

// out = C_m X C_n^T (forward) or C_m^T X C_n (transposed); tmp: m x n.
cudaError_t dct2(const cpa_completion_ctx *c, const float *X, int64_t ldx, bool transposed, float *tmp, float *out,
                 cudaStream_t st, bool tc) {
    if (tc) return dct2_tc(c, X, ldx, transposed, tmp, out, st);
    const int m = (int)c->m, n = (int)c->n;
    Epilogue e1;
    e1.D = tmp;
    e1.ldd = n;
    Epilogue e2;
    e2.D = out;
    e2.ldd = n;
    cudaError_t r;
    if (!transposed) {
        // tmp(i,j) = sum_k X(i,k) C_n(j,k);  out(i,j) = sum_k C_m(i,k) tmp(k,j)
        if ((r = gemm_f32(m, n, n, X, ldx, true, c->Cn, n, true, e1, st)) != cudaSuccess) return r;
        return gemm_f32(m, n, m, c->Cm, m, true, tmp, n, false, e2, st);
    }
    // tmp(i,j) = sum_k X(i,k) C_n(k,j);  out(i,j) = sum_k C_m(k,i) tmp(k,j)
    if ((r = gemm_f32(m, n, n, X, ldx, true, c->Cn, n, false, e1, st)) != cudaSuccess) return r;
    return gemm_f32(m, n, m, c->Cm, m, false, tmp, n, false, e2, st);
}
}  // namespace

extern "C" {

cpa_status cpa_completion_create(cpa_handle h, int64_t m, int64_t n, cpa_completion *out) {
    if (!h || !out || m < 1 || n < 1 || m > 65536 || n > 65536 || m * n > ((int64_t)1 << 31))
        return CPA_ERR_INVALID_ARG;
    *out = nullptr;
    cpa_completion c = new cpa_completion_ctx();
    c->h = h;
    c->m = m;
    c->n = n;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return CPA_ERR_CUDA;
    }
    if (cudaMalloc(&c->Cm, sizeof(float) * (size_t)(m * m)) != cudaSuccess ||
        cudaMalloc(&c->Cn, sizeof(float) * (size_t)(n * n)) != cudaSuccess ||
        cudaMalloc(&c->state, sizeof(float) * 10 * (size_t)(m * n)) != cudaSuccess) {
        cudaFree(c->Cm);
        cudaFree(c->Cn);
        cudaFree(c->state);
        delete c;
        return CPA_ERR_NO_MEMORY;
    }
    c->bm = (m + 7) / 8 * 8;
    c->bn = (n + 7) / 8 * 8;
    const size_t nb = 4 * (size_t)(m * c->bm) + 4 * (size_t)(n * c->bn) + 2 * (size_t)(m * c->bn) +
                      2 * (size_t)(n * c->bm) + 64;
    if (cudaMalloc(&c->bf, sizeof(__nv_bfloat16) * nb) != cudaSuccess) {
        cudaFree(c->Cm);
        cudaFree(c->Cn);
        cudaFree(c->state);
        delete c;
        return CPA_ERR_NO_MEMORY;
    }
    // pieces 16-byte aligned: every size is a multiple of 8 elements
    __nv_bfloat16 *q = c->bf;
    auto take = [&](size_t count) {
        __nv_bfloat16 *r = q;
        q += count;
        return r;
    };
    c->Cmh = take(m * c->bm);
    c->Cml = take(m * c->bm);
    c->CmTh = take(m * c->bm);
    c->CmTl = take(m * c->bm);
    c->Cnh = take(n * c->bn);
    c->Cnl = take(n * c->bn);
    c->CnTh = take(n * c->bn);
    c->CnTl = take(n * c->bn);
    c->Xh = take(m * c->bn);
    c->Xl = take(m * c->bn);
    c->Th = take(n * c->bm);
    c->Tl = take(n * c->bm);
    float *tab = nullptr;   // the DCT's cosine table (4 max(m, n) floats), freed below
    if (cudaMalloc(&tab, sizeof(float) * 4 * (size_t)std::max(m, n)) != cudaSuccess ||
        make_transform(CPA_T_DCT, (int)m, c->Cm, m, 0, c->num_sms, tab) != cudaSuccess ||
        make_transform(CPA_T_DCT, (int)n, c->Cn, n, 0, c->num_sms, tab) != cudaSuccess ||
        split_bf16(c->Cm, (int)m, (int)m, m, false, c->Cmh, c->Cml, c->bm, 0) != cudaSuccess ||
        split_bf16(c->Cm, (int)m, (int)m, m, true, c->CmTh, c->CmTl, c->bm, 0) != cudaSuccess ||
        split_bf16(c->Cn, (int)n, (int)n, n, false, c->Cnh, c->Cnl, c->bn, 0) != cudaSuccess ||
        split_bf16(c->Cn, (int)n, (int)n, n, true, c->CnTh, c->CnTl, c->bn, 0) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        if (tab) cudaFree(tab);
        cudaFree(c->Cm);
        cudaFree(c->Cn);
        cudaFree(c->state);
        cudaFree(c->bf);
        delete c;
        return CPA_ERR_CUDA;
    }
    cudaFree(tab);
    *out = c;
    return CPA_OK;
}

cpa_status cpa_completion_destroy(cpa_completion c) {
    if (!c) return CPA_ERR_INVALID_ARG;
    cudaFree(c->Cm);
    cudaFree(c->Cn);
    cudaFree(c->state);
    cudaFree(c->acc);
    cudaFree(c->bf);
    delete c;
    return CPA_OK;
}

cpa_status cpa_completion_run(cpa_completion c, const float *dI, int64_t ldi, const uint8_t *dmask, int64_t ldmask,
                              double tau_nuclear, double tau_l1, int L, int prec, int max_iters, double tol,
                              float *dL, int64_t ldl, float *dZ1, int *iters_done, double *errors, void *stream) {
    if (!c || !dI || !dmask || !dL || ldi < c->n || ldmask < c->n || ldl < c->n || !(tau_nuclear >= 0.0) ||
        !(tau_l1 >= 0.0) || !std::isfinite(tau_nuclear) || !std::isfinite(tau_l1) || L < 1 || max_iters < 1 ||
        !(tol >= 0.0))
        return CPA_ERR_INVALID_ARG;
    const int64_t m = c->m, n = c->n, total = m * n;
    auto overlap = [](const void *p, size_t pb, const void *q, size_t qb) {
        const uintptr_t x = (uintptr_t)p, y = (uintptr_t)q;
        return x < y + qb && y < x + pb;
    };
    const size_t lb = sizeof(float) * (size_t)((m - 1) * ldl + n), ib = sizeof(float) * (size_t)((m - 1) * ldi + n);
    const size_t mb = (size_t)((m - 1) * ldmask + n), zb = sizeof(float) * (size_t)total;
    if (overlap(dL, lb, dI, ib) || overlap(dL, lb, dmask, mb) || (dZ1 && (overlap(dZ1, zb, dL, lb) ||
                                                                          overlap(dZ1, zb, dI, ib) ||
                                                                          overlap(dZ1, zb, dmask, mb))))
        return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(c->device) != cudaSuccess) return CPA_ERR_CUDA;
    if (c->acc_cap < max_iters) {
        cudaFree(c->acc);
        c->acc = nullptr;
        if (cudaMalloc(&c->acc, sizeof(double) * 2 * (size_t)max_iters) != cudaSuccess) return CPA_ERR_NO_MEMORY;
        c->acc_cap = max_iters;
    }
    float *u1 = c->state, *u2 = u1 + total, *u3 = u2 + total, *u4 = u3 + total, *S = u4 + total, *A2 = S + total,
          *W = A2 + total, *Z1 = W + total, *T1 = Z1 + total, *T2 = T1 + total;
    const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, (int64_t)c->num_sms * 8);
    cpa_status r;
    if ((r = ccuda(cudaMemsetAsync(c->acc, 0, sizeof(double) * 2 * (size_t)max_iters, st))) != CPA_OK) return r;
    init_kernel<<<blocks, kThreads, 0, st>>>((int)m, (int)n, dL, ldl, u1, u2, u3, u4, S);
    if ((r = ccuda(cudaGetLastError())) != CPA_OK) return r;
    // z_0 = K l_0 with l_0 = 1: a2 = Psi 1 - 1
    const bool tc = prec != CPA_FP32;
    if ((r = ccuda(dct2(c, dL, ldl, false, T1, T2, st, tc))) != CPA_OK) return r;
    init_a2_kernel<<<blocks, kThreads, 0, st>>>(total, T2, A2);
    if ((r = ccuda(cudaGetLastError())) != CPA_OK) return r;
    cpa_shrink sh{};
    sh.kind = CPA_SOFT;
    sh.tau = tau_nuclear;
    int done = 0;
    for (int t = 0; t < max_iters; ++t) {
        // least-squares step: l = (S + Psi^T A2) / (3 + omega)
        if ((r = ccuda(dct2(c, A2, n, true, T1, T2, st, tc))) != CPA_OK) return r;
        ls_kernel<<<blocks, kThreads, 0, st>>>((int)m, (int)n, dmask, ldmask, S, T2, u1, dL, ldl, W, c->acc + 2 * t);
        if ((r = ccuda(cudaGetLastError())) != CPA_OK) return r;
        // z1 = prox_{(1/rho)|.|_*}(l + u1): Algorithm 1, Lambda_max computed
        if ((r = cpa_svt(c->h, W, m, n, n, &sh, L, 0.0, prec, nullptr, Z1, n, stream)) != CPA_OK) return r;
        // P = Psi l, then the z and u updates
        if ((r = ccuda(dct2(c, dL, ldl, false, T1, T2, st, tc))) != CPA_OK) return r;
        update_kernel<<<blocks, kThreads, 0, st>>>((int)m, (int)n, dI, ldi, dmask, ldmask, dL, ldl, Z1, T2, u1, u2,
                                                   u3, u4, A2, S, (float)tau_l1);
        if ((r = ccuda(cudaGetLastError())) != CPA_OK) return r;
        done = t + 1;
        if (tol > 0.0) {
            double e2[2];
            if ((r = ccuda(cudaMemcpyAsync(e2, c->acc + 2 * t, sizeof e2, cudaMemcpyDeviceToHost, st))) != CPA_OK)
                return r;
            if ((r = ccuda(cudaStreamSynchronize(st))) != CPA_OK) return r;
            if (e2[1] > 0.0 && std::sqrt(e2[0] / e2[1]) < tol) break;
        }
    }
    if (dZ1 && (r = ccuda(cudaMemcpyAsync(dZ1, Z1, sizeof(float) * (size_t)total, cudaMemcpyDeviceToDevice, st))) !=
                   CPA_OK)
        return r;
    if (iters_done) *iters_done = done;
    if (errors) {
        std::vector<double> e2(2 * (size_t)done);
        if ((r = ccuda(cudaMemcpyAsync(e2.data(), c->acc, sizeof(double) * e2.size(), cudaMemcpyDeviceToHost, st))) !=
            CPA_OK)
            return r;
        if ((r = ccuda(cudaStreamSynchronize(st))) != CPA_OK) return r;
        for (int t = 0; t < done; ++t) errors[t] = e2[2 * t + 1] > 0.0 ? std::sqrt(e2[2 * t] / e2[2 * t + 1]) : 0.0;
    }
    return CPA_OK;
}

}  // extern "C"
