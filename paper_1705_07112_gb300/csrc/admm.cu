// Background-modelling ADMM (the appendix ADMM Applicable Forms, Background Modeling, Eq. admm_algorithm_mod) around the
// CPA shrinkage: min |l|_* + eta |s|_1 subject to l + s = d, written with
// z = K l', K = [[I, 0], [0, I], [I, I]] and solved by ADMM.  Iteration t:
//   l', s' = (K^T K)^{-1} K^T (z - u)           (closed form below)
//   z1 = prox_{(1/rho)|.|_*}(l + u1)            cpa_svt, soft, tau = 1/rho
//   z2 = prox_{(eta/rho)|.|_1}(s + u2)          entrywise soft threshold
//   z3 = d                                      projection onto {x = d}
//   u += K l' - z
// With a_i = z_i - u_i:  l = (2 a1 - a2 + a3) / 3,  s = (-a1 + 2 a2 + a3) / 3.
// Start (Section V, Background Modeling of Video): l = s = u = 1, z = K l'.
//
// Device state: l, s, u1, u2, u3 and the next shrinkage input w = l + u1
// (FP32, m x n, owned by the solver object); z1 lives in the caller's L
// output and z2 in its S output.  One fused kernel per iteration finishes
// iteration t (z2, u) and starts t + 1 (l, s, w, and the sums of
// E_{t+1} = |l_{t+1} - l_t|_F / |l_{t+1}|_F, the stopping quantity of
// the stopping-criterion footnote of Section V, Optimization Tools).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.h"

namespace cpa {
namespace {

constexpr int kAdmmThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float soft1(float x, float t) {
    const float a = fabsf(x) - t;
    return a > 0.f ? copysignf(a, x) : 0.f;
}

// l = s = 1/3, u = 1, w = 4/3: the first least-squares step from the
// all-ones start (a = z - u = (0, 0, 1)).
__global__ void admm_init_kernel(int64_t total, float *l, float *s, float *u1, float *u2, float *u3, float *w) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        l[e] = 1.f / 3.f;
        s[e] = 1.f / 3.f;
        u1[e] = 1.f;
        u2[e] = 1.f;
        u3[e] = 1.f;
        w[e] = 1.f / 3.f + 1.f;
    }
}

// Finishes iteration t given z1 (the shrinkage of w) and starts t + 1.
// acc[0] += |l_{t+1} - l_t|^2, acc[1] += |l_{t+1}|^2 (FP64, one atomic per
// warp).
__global__ void __launch_bounds__(kAdmmThreads)
    admm_step_kernel(const float *__restrict__ D, int64_t ldd, int m, int n, float *__restrict__ l,
                     float *__restrict__ s, float *__restrict__ u1, float *__restrict__ u2, float *__restrict__ u3,
                     float *__restrict__ w, const float *__restrict__ z1, float *__restrict__ z2, float tau_l1,
                     double *__restrict__ acc) {
    const int64_t total = (int64_t)m * n;
    double dsum = 0.0, lsum = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        const float d = __ldg(D + i * ldd + j);
        const float le = l[e], se = s[e];
        float a = u1[e], b = u2[e], c = u3[e];
        const float y1 = z1[e];
        const float y2 = soft1(se + b, tau_l1);
        a += le - y1;            // u_{t+1} = u_t + K l'_{t+1} - z_{t+1}
        b += se - y2;
        c += le + se - d;
        const float a1 = y1 - a, a2 = y2 - b, a3 = d - c;
        const float ln = (2.f * a1 - a2 + a3) * (1.f / 3.f);
        const float sn = (-a1 + 2.f * a2 + a3) * (1.f / 3.f);
        const double dl = (double)ln - (double)le;
        dsum += dl * dl;
        lsum += (double)ln * (double)ln;
        l[e] = ln;
        s[e] = sn;
        u1[e] = a;
        u2[e] = b;
        u3[e] = c;
        w[e] = ln + a;
        z2[e] = y2;
    }
    dsum = warp_sum_d(dsum);
    lsum = warp_sum_d(lsum);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, dsum);
        atomicAdd(acc + 1, lsum);
    }
}

}  // namespace
}  // namespace cpa

using namespace cpa;

struct cpa_admm_ctx {
    cpa_handle h = nullptr;
    int device = 0;
    int num_sms = 0;
    int64_t m = 0, n = 0;
    float *state = nullptr;     // l, s, u1, u2, u3, w: 6 m n floats
    double *acc = nullptr;      // 2 doubles per iteration
    int acc_cap = 0;
};

namespace {
cpa_status admm_cuda(cudaError_t e) { return e == cudaSuccess ? CPA_OK : CPA_ERR_CUDA; }
}  // namespace

extern "C" {

cpa_status cpa_admm_create(cpa_handle h, int64_t m, int64_t n, cpa_admm *out) {
    if (!h || !out || m < 1 || n < 1 || m * n > ((int64_t)1 << 31)) return CPA_ERR_INVALID_ARG;
    *out = nullptr;
    cpa_admm a = new cpa_admm_ctx();
    a->h = h;
    a->m = m;
    a->n = n;
    if (cudaGetDevice(&a->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&a->num_sms, cudaDevAttrMultiProcessorCount, a->device) != cudaSuccess) {
        delete a;
        return CPA_ERR_CUDA;
    }
    if (cudaMalloc(&a->state, sizeof(float) * 6 * (size_t)(m * n)) != cudaSuccess) {
        delete a;
        return CPA_ERR_NO_MEMORY;
    }
    *out = a;
    return CPA_OK;
}

cpa_status cpa_admm_destroy(cpa_admm a) {
    if (!a) return CPA_ERR_INVALID_ARG;
    cudaFree(a->state);
    cudaFree(a->acc);
    delete a;
    return CPA_OK;
}

cpa_status cpa_admm_rpca(cpa_admm a, const float *dD, int64_t ldd, double tau_nuclear, double tau_l1, int L,
                         int prec, const cpa_sparsify *sp, int schedule, int max_iters, double tol, float *dL,
                         float *dS, int *iters_done, double *errors, void *stream) {
    if (!a || !dD || !dL || !dS || ldd < a->n || !(tau_nuclear >= 0.0) || !(tau_l1 >= 0.0) || L < 1 ||
        max_iters < 1 || !(tol >= 0.0) || !std::isfinite(tau_nuclear) || !std::isfinite(tau_l1))
        return CPA_ERR_INVALID_ARG;
    if (schedule && (!sp || sp->mode != CPA_SPARSE_TOPK)) return CPA_ERR_INVALID_ARG;
    const int64_t m = a->m, n = a->n, total = m * n;
    // outputs must not overlap the input or each other
    auto overlap = [](const void *p, size_t pb, const void *q, size_t qb) {
        const uintptr_t x = (uintptr_t)p, y = (uintptr_t)q;
        return x < y + qb && y < x + pb;
    };
    const size_t ob = sizeof(float) * (size_t)total, db = sizeof(float) * (size_t)((m - 1) * ldd + n);
    if (overlap(dL, ob, dS, ob) || overlap(dL, ob, dD, db) || overlap(dS, ob, dD, db)) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(a->device) != cudaSuccess) return CPA_ERR_CUDA;
    if (a->acc_cap < max_iters) {
        cudaFree(a->acc);
        a->acc = nullptr;
        if (cudaMalloc(&a->acc, sizeof(double) * 2 * (size_t)max_iters) != cudaSuccess) return CPA_ERR_NO_MEMORY;
        a->acc_cap = max_iters;
    }
    float *l = a->state, *s = l + total, *u1 = s + total, *u2 = u1 + total, *u3 = u2 + total, *w = u3 + total;
    const int blocks = (int)std::min<int64_t>((total + kAdmmThreads - 1) / kAdmmThreads, (int64_t)a->num_sms * 8);
    cpa_status r;
    if ((r = admm_cuda(cudaMemsetAsync(a->acc, 0, sizeof(double) * 2 * (size_t)max_iters, st))) != CPA_OK) return r;
    admm_init_kernel<<<blocks, kAdmmThreads, 0, st>>>(total, l, s, u1, u2, u3, w);
    if ((r = admm_cuda(cudaGetLastError())) != CPA_OK) return r;
    cpa_shrink sh{};
    sh.kind = CPA_SOFT;
    sh.tau = tau_nuclear;
    int done = 0;
    cpa_sparsify spt{};
    if (sp) spt = *sp;
    for (int t = 0; t < max_iters; ++t) {
        if (schedule) {
            // the current E_t picks the kept fraction (Eq. recommendation_epsilon);
            // the start l_1 = 1/3 after l_0 = 1 has E = 2
            double E = 2.0;
            if (t > 0) {
                double e2[2];
                if ((r = admm_cuda(cudaMemcpyAsync(e2, a->acc + 2 * (t - 1), sizeof e2, cudaMemcpyDeviceToHost,
                                                   st))) != CPA_OK)
                    return r;
                if ((r = admm_cuda(cudaStreamSynchronize(st))) != CPA_OK) return r;
                E = e2[1] > 0.0 ? std::sqrt(e2[0] / e2[1]) : 0.0;
            }
            spt.eps_or_frac = E > 0.3e-1 ? 0.5e-4 : (E > 6e-4 ? 1.5e-4 : 0.5e-3);
        }
        // z1 = prox_{(1/rho)|.|_*}(l + u1): Algorithm 1, Lambda_max computed
        if ((r = cpa_svt(a->h, w, m, n, n, &sh, L, 0.0, prec, sp ? &spt : nullptr, dL, n, stream)) != CPA_OK)
            return r;
        admm_step_kernel<<<blocks, kAdmmThreads, 0, st>>>(dD, ldd, (int)m, (int)n, l, s, u1, u2, u3, w, dL, dS,
                                                          (float)tau_l1, a->acc + 2 * t);
        if ((r = admm_cuda(cudaGetLastError())) != CPA_OK) return r;
        done = t + 1;
        if (tol > 0.0) {
            double e2[2];
            if ((r = admm_cuda(cudaMemcpyAsync(e2, a->acc + 2 * t, sizeof e2, cudaMemcpyDeviceToHost, st))) !=
                CPA_OK)
                return r;
            if ((r = admm_cuda(cudaStreamSynchronize(st))) != CPA_OK) return r;
            if (e2[1] > 0.0 && std::sqrt(e2[0] / e2[1]) < tol) break;
        }
    }
    if (iters_done) *iters_done = done;
    if (errors) {
        std::vector<double> e2(2 * (size_t)done);
        if ((r = admm_cuda(cudaMemcpyAsync(e2.data(), a->acc, sizeof(double) * e2.size(), cudaMemcpyDeviceToHost,
                                           st))) != CPA_OK)
            return r;
        if ((r = admm_cuda(cudaStreamSynchronize(st))) != CPA_OK) return r;
        for (int t = 0; t < done; ++t) errors[t] = e2[2 * t + 1] > 0.0 ? std::sqrt(e2[2 * t] / e2[2 * t + 1]) : 0.0;
    }
    return CPA_OK;
}

}  // extern "C"
