// Learned choice of (Lambda_max, L) for one matrix of any size, inside the
// single-matrix shrinkage.  The paper has no counterpart: the predictor
// network picks the interval bound and the order of Algorithm 1 from cheap
// features of the Gram matrix, so that each matrix gets the fewest terms
// that reach the error it was trained for.
//
// learn_bound_kernel (one cooperative launch, grid barriers between its
// phases, one warp per row of G, rows grid-strided):
//   1. power products w_t = G v_{t-1} / |v_{t-1}| from the SplitMix64 start
//      vector, t = 1..T (T = 5 with the predicted bound, iters + 1
//      without), with theta_t = v_hat_{t-1} . w_t and |w_t|^2 summed in FP64
//      across blocks; the residual |w_t - theta_t v_hat_{t-1}| at t = 4 and
//      t = T; the trace and |G|_F^2 during the first product;
//   2. the lower spectral edge: four steps u <- (theta_4 I - G) u / |.| from
//      a second SplitMix64 vector, then lambda_min = u.Gu / u.u;
//   3. block 0: the twelve features (the definition of cpa_batch_features),
//      the 12 -> 64 -> 64 -> 2 network in the summation order of the
//      network's own forward kernel, and the decision rule of
//      cpa_svt_batched_learned; writes {theta, r, trace, lambda, status} and
//      L to the device;
//   4. every block: a slice of the table cos(pi m / 2L) (m = 0..L) and of the
//      response at the L nodes, then, after a barrier, a slice of the
//      coefficients of Eq. chebychev_coeff_shifted (FP64); c_k = 0 for
//      L <= k < L_max so that later kernels may read L_max of them.
// The recurrence then reads L from the device (gemm_tc_recurrence's L_dev),
// so the whole call stays asynchronous.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace cpa {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kFeat = 12, kHid = 64;
constexpr uint64_t kEdgeSeedXor = 0x5EEDULL;   // start vector of the lower-edge steps

__device__ __forceinline__ uint64_t splitmix64_l(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float start_value(uint64_t seed, int i) {
    const uint64_t z = splitmix64_l(seed, (uint64_t)i);
    return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid barrier (monotone counter zeroed before the launch, bounded wait:
// on expiry CPA_ERR_TIMEOUT in *err and the block goes on).
__device__ __forceinline__ void lgrid_barrier(unsigned int *count, unsigned int &target, int *err, long long limit,
                                              unsigned int extra = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x + extra;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        const long long t0 = clock64();
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > limit) {
                atomicExch(err, (int)CPA_ERR_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();
}

// Block sums of up to three floats (one per warp lane 0 partial), added to
// FP64 slots by one atomic each.
struct Partials {
    float a[kWarps], b[kWarps], c[kWarps];
};
__device__ __forceinline__ void block_add(Partials &sh, float a, float b, float c, double *sa, double *sb,
                                          double *sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh.a[w] = a;
        sh.b[w] = b;
        sh.c[w] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < kWarps ? sh.a[threadIdx.x] : 0.f;
        float y = threadIdx.x < kWarps ? sh.b[threadIdx.x] : 0.f;
        float z = threadIdx.x < kWarps ? sh.c[threadIdx.x] : 0.f;
        x = warp_sum_f(x);
        y = warp_sum_f(y);
        z = warp_sum_f(z);
        if (threadIdx.x == 0) {
            if (sa && x != 0.f) atomicAdd(sa, (double)x);
            if (sb && y != 0.f) atomicAdd(sb, (double)y);
            if (sc && z != 0.f) atomicAdd(sc, (double)z);
        }
    }
    __syncthreads();
}

struct LearnRule {
    const float *P;      // network parameters: W1[64][12], b1, W2[64][64], b2, W3[2][64], b3
    double L_scale, margin;
    int L_min, L_max, L_fallback, use_lambda;
    int feat_only;
};

// FP64 accumulator slots (zeroed by block 0 before the first barrier).
enum Slot {
    kNrm = 0,                       // |w_t|^2, t = 0..T (t = 0: the start vector)
    kDot = kNrm + 32,               // theta_t, t = 1..T
    kR4 = kDot + 32,                // residual^2 at t = 4
    kRT,                            // residual^2 at t = T
    kFro, kTr,                      // |G|_F^2, trace
    kUn,                            // lower edge: |u_s|^2, s = 0..4 (5 slots)
    kUnum = kUn + 5, kUden,         // u.Gu, u.u
    kSlots
};

__global__ void __launch_bounds__(kThreads) learn_bound_kernel(
    const float *__restrict__ G, int64_t ldg, int p, int q, ShrinkParams sp, LearnRule rule, int iters,
    float *v0, float *v1, float *u0, float *u1, double *acc, unsigned int *bar, int *err, double *out, int *L_out,
    float *feat, double *theta_out, double *coef, double *tabg, long long wait, int stall) {
    extern __shared__ __align__(16) unsigned char lsm[];
    float *vs = reinterpret_cast<float *>(lsm);   // staged iterate (when it fits)
    __shared__ Partials part;
    __shared__ float fv[kFeat];
    __shared__ float h1s[kHid], h2s[kHid], ys[2];
    unsigned int target = 0;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kThreads) >> 5;
    const int its = (rule.use_lambda || rule.feat_only) ? 4 : iters;
    const int T = its + 1;   // products of the main iteration
    const int p4 = (p + 3) & ~3;
    const bool stage = (size_t)p4 * sizeof(float) <= 96 * 1024;

    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < kSlots; i += kThreads) acc[i] = 0.0;
        __syncthreads();
        float s = 0.f, su = 0.f;
        for (int i = threadIdx.x; i < p4; i += kThreads) {
            const float x = i < p ? start_value(kStartSeed, i) : 0.f;
            const float y = i < p ? start_value(kStartSeed ^ kEdgeSeedXor, i) : 0.f;
            v0[i] = x;
            v1[i] = 0.f;
            u0[i] = y;
            u1[i] = 0.f;
            s = fmaf(x, x, s);
            su = fmaf(y, y, su);
        }
        s = warp_sum_f(s);
        su = warp_sum_f(su);
        block_add(part, s, su, 0.f, acc + kNrm, acc + kUn, nullptr);
    }
    lgrid_barrier(bar, target, err, wait, stall ? 1u : 0u);

    // ---- main power iteration: product t reads v_{t-1} (buffer (t-1)&1),
    // writes w_t (buffer t&1, the next iterate, unnormalised)
    for (int t = 1; t <= T; ++t) {
        const float *v = ((t - 1) & 1) ? v1 : v0;
        float *w = (t & 1) ? v1 : v0;
        const double nin = __ldcg(&acc[kNrm + t - 1]);
        const float sc = nin > 0.0 ? __frcp_rn(__fsqrt_rn((float)nin)) : 0.f;
        // residual of the previous product (t - 1 = 4): its rows are the
        // ones this warp writes now, w_{t-1} lives in buffer (t-1)&1 = v,
        // v_{t-2} in buffer t&1 = w (not yet overwritten for these rows)
        const bool res4 = (t - 1 == 4);
        const double th_prev = res4 ? __ldcg(&acc[kDot + 4]) : 0.0;
        const double nprev = res4 ? __ldcg(&acc[kNrm + 3]) : 0.0;
        const float scp = nprev > 0.0 ? __frcp_rn(__fsqrt_rn((float)nprev)) : 0.f;
        if (stage) {
            const float4 *src = reinterpret_cast<const float4 *>(v);
            float4 *dst = reinterpret_cast<float4 *>(vs);
            for (int i = threadIdx.x; i < (p4 >> 2); i += kThreads) dst[i] = __ldcg(src + i);
            __syncthreads();
        }
        const float *vsrc = stage ? vs : v;
        float pn = 0.f, pd = 0.f, pr = 0.f, pf = 0.f, ptr = 0.f;
        for (int row = gwarp; row < p; row += nwarps) {
            const float *g = G + (int64_t)row * ldg;
            float a = 0.f, f2 = 0.f;
            for (int j = lane; j < p; j += 32) {
                const float gv = __ldg(g + j);
                a = fmaf(gv, stage ? vsrc[j] : __ldcg(vsrc + j), a);
                if (t == 1) f2 = fmaf(gv, gv, f2);
            }
            a = warp_sum_f(a) * sc;
            if (t == 1) f2 = warp_sum_f(f2);
            if (lane == 0) {
                const float vr = stage ? vsrc[row] : __ldcg(vsrc + row);
                if (res4) {
                    // w_4 = v (this product's input), v_hat_3 = (buffer t&1) * scp
                    const float d = vr - (float)th_prev * __ldcg(w + row) * scp;
                    pr = fmaf(d, d, pr);
                }
                w[row] = a;
                pn = fmaf(a, a, pn);
                pd = fmaf(vr * sc, a, pd);
                if (t == 1) {
                    pf += f2;
                    ptr += __ldg(g + row);
                }
            }
        }
        block_add(part, pn, pd, pr, acc + kNrm + t, acc + kDot + t, res4 ? acc + kR4 : nullptr);
        if (t == 1) block_add(part, pf, ptr, 0.f, acc + kFro, acc + kTr, nullptr);
        lgrid_barrier(bar, target, err, wait);
    }
    // residual of the last product: w_T in buffer T&1, v_{T-1} in (T-1)&1
    {
        const float *wT = (T & 1) ? v1 : v0;
        const float *vp = ((T - 1) & 1) ? v1 : v0;
        const double th = __ldcg(&acc[kDot + T]);
        const double nprev = __ldcg(&acc[kNrm + T - 1]);
        const float scp = nprev > 0.0 ? __frcp_rn(__fsqrt_rn((float)nprev)) : 0.f;
        float pr = 0.f;
        for (int row = gwarp; row < p; row += nwarps)
            if (lane == 0) {
                const float d = __ldcg(wT + row) - (float)th * __ldcg(vp + row) * scp;
                pr = fmaf(d, d, pr);
            }
        block_add(part, pr, 0.f, 0.f, acc + kRT, nullptr, nullptr);
    }
    // ---- lower spectral edge: u <- (theta_4 u - G u) / |.|, four steps,
    // then lambda_min = u.Gu / u.u (step s reads u_s from buffer s&1)
    const float th4f = (float)__ldcg(&acc[kDot + 4]);
    for (int sidx = 0; sidx <= 4; ++sidx) {
        const float *u = (sidx & 1) ? u1 : u0;
        float *un = (sidx & 1) ? u0 : u1;
        // the previous step's vector and norm are complete in every block
        lgrid_barrier(bar, target, err, wait);
        const double nin = __ldcg(&acc[kUn + sidx]);
        const float sc = sidx == 0 ? 1.f : (nin > 0.0 ? __frcp_rn(__fsqrt_rn((float)nin)) : 0.f);
        if (stage) {
            const float4 *src = reinterpret_cast<const float4 *>(u);
            float4 *dst = reinterpret_cast<float4 *>(vs);
            for (int i = threadIdx.x; i < (p4 >> 2); i += kThreads) dst[i] = __ldcg(src + i);
            __syncthreads();
        }
        const float *usrc = stage ? vs : u;
        float pa = 0.f, pb = 0.f;
        for (int row = gwarp; row < p; row += nwarps) {
            const float *g = G + (int64_t)row * ldg;
            float a = 0.f;
            for (int j = lane; j < p; j += 32) a = fmaf(__ldg(g + j), stage ? usrc[j] : __ldcg(usrc + j), a);
            a = warp_sum_f(a) * sc;   // G u_hat (the stored u is unnormalised)
            if (lane == 0) {
                const float ur = (stage ? usrc[row] : __ldcg(usrc + row)) * sc;
                if (sidx < 4) {
                    const float nx = th4f * ur - a;
                    un[row] = nx;
                    pa = fmaf(nx, nx, pa);
                } else {
                    pa = fmaf(ur, a, pa);
                    pb = fmaf(ur, ur, pb);
                }
            }
        }
        if (sidx < 4)
            block_add(part, pa, 0.f, 0.f, acc + kUn + sidx + 1, nullptr, nullptr);
        else
            block_add(part, pa, pb, 0.f, acc + kUnum, acc + kUden, nullptr);
    }
    lgrid_barrier(bar, target, err, wait);

    // ---- features, network and decision (block 0)
    if (blockIdx.x == 0) {
        const int tid = threadIdx.x;
        const double E0 = __ldcg(&acc[kTr]);
        const double E = E0 > 0.0 ? E0 : 1.0;
        const double tiny = 1e-30;
        const double th2 = __ldcg(&acc[kDot + 2]), th4 = __ldcg(&acc[kDot + 4]);
        const double r4 = sqrt(fmax(__ldcg(&acc[kR4]), 0.0));
        const double den = __ldcg(&acc[kUden]);
        const double lmin = den > 0.0 ? __ldcg(&acc[kUnum]) / den : 0.0;
        const double fro = __ldcg(&acc[kFro]);
        if (tid < kFeat) {
            const double t4 = fmax(th4, tiny * E);
            double thr2;
            if (sp.kind == CPA_WSOFT) {
                const double se = sqrt(fmax(th4 - sp.noise, 0.0));
                const double wv = sp.c / (se + sp.eps);
                thr2 = wv * wv;
            } else {
                thr2 = sp.tau * sp.tau;
            }
            thr2 = fmax(thr2, tiny * E);
            const double lm = fmax(lmin, tiny * E);
            double r = 1.0;
            switch (tid) {
                case 0: r = (double)p; break;
                case 1: r = (double)q / (double)p; break;
                case 2: r = E / t4; break;
                case 3: r = thr2 / t4; break;
                case 4: r = lm / t4; break;
                case 5: r = thr2 / lm; break;
                case 6: r = fmax(fro, tiny * E * E) / (t4 * t4); break;
                case 7: r = E / ((double)p * thr2); break;
                case 8: r = t4 / fmax(th2, tiny * E); break;
                case 9: r = (t4 + r4) / t4; break;
                default: break;
            }
            fv[tid] = tid == 10 ? (sp.kind == CPA_HARD ? 1.f : 0.f)
                      : tid == 11 ? (sp.kind == CPA_WSOFT ? 1.f : 0.f)
                                  : logf((float)r);
        }
        __syncthreads();
        if (rule.feat_only) {
            if (tid < kFeat) feat[tid] = fv[tid];
            if (tid == 0) {
                theta_out[0] = th4;
                out[4] = (isfinite(E0) && isfinite(fro)) ? 0.0 : (double)CPA_ERR_NONFINITE;
                const int e2 = __ldcg(err);
                if (e2) out[4] = (double)e2;
            }
        } else {
            const float *P = rule.P;
            constexpr int oW1 = 0, ob1 = kHid * kFeat, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid,
                          oW3 = ob2 + kHid, ob3 = oW3 + 2 * kHid;
            if (tid < kHid) {
                float a = __ldg(P + ob1 + tid);
                for (int j = 0; j < kFeat; ++j) a = fmaf(__ldg(P + oW1 + tid * kFeat + j), fv[j], a);
                h1s[tid] = a > 0.f ? a : 0.f;
            }
            __syncthreads();
            if (tid < kHid) {
                float a = __ldg(P + ob2 + tid);
                for (int j = 0; j < kHid; ++j) a = fmaf(__ldg(P + oW2 + tid * kHid + j), h1s[j], a);
                h2s[tid] = a > 0.f ? a : 0.f;
            }
            __syncthreads();
            if (tid < 2) {
                float a = __ldg(P + ob3 + tid);
                for (int j = 0; j < kHid; ++j) a = fmaf(__ldg(P + oW3 + tid * kHid + j), h2s[j], a);
                ys[tid] = a;
            }
            __syncthreads();
            if (tid == 0) {
                // the power bound of the main iteration's last product
                const double thT = __ldcg(&acc[kDot + T]);
                const double rT = sqrt(fmax(__ldcg(&acc[kRT]), 0.0));
                double lb = (thT + rT) * (1.0 + kLambdaMargin);
                if (lb > E0) lb = E0;
                double status = 0.0;
                if (!isfinite(lb) || !isfinite(E0) || !isfinite(fro)) {
                    status = (double)CPA_ERR_NONFINITE;
                    lb = 1.0;
                } else if (!(lb > 0.0)) {
                    lb = E0 > 0.0 ? E0 : 1.0;
                }
                const double y0 = (double)ys[0], y1 = (double)ys[1];
                const double Lf = ceil(exp(y1) * rule.L_scale);
                const bool ok_L = isfinite(Lf) && Lf <= (double)rule.L_max;
                int Lc = ok_L ? (int)Lf : rule.L_fallback;
                if (Lc < rule.L_min) Lc = rule.L_min;
                double lc = lb;
                bool ok_lam = true;
                if (rule.use_lambda) {
                    const double lp = th4 * exp(fmax(y0, 0.0)) * (1.0 + rule.margin);
                    const double floor_lam = (th4 + r4) * (1.0 + kLambdaMargin);
                    ok_lam = isfinite(lp) && lp > 0.0;
                    if (isfinite(lp) && lp > 0.0 && isfinite(floor_lam))
                        lc = fmax(lp, floor_lam);
                    else
                        Lc = rule.L_fallback;
                }
                if (!(lc > 0.0) || !isfinite(lc)) lc = lb;
                const int e2 = __ldcg(err);
                if (e2) status = (double)e2;
                out[0] = thT;
                out[1] = rT;
                out[2] = E0;
                out[3] = lc;
                out[4] = status;
                L_out[0] = Lc;
                L_out[1] = (!ok_L || !ok_lam) ? 1 : 0;
                tabg[0] = lc;   // broadcast to the other blocks
                reinterpret_cast<int *>(tabg)[2] = Lc;
            }
            __syncthreads();
        }
    }
    if (rule.feat_only) return;
    lgrid_barrier(bar, target, err, wait);
    // ---- coefficients on [0, lambda] for the chosen L
    const double lam = __ldcg(&tabg[0]);
    const int L = __ldcg(reinterpret_cast<const int *>(tabg) + 2);
    double *tab = tabg + 2;            // cos(pi m / 2L), m = 0..L
    double *hs = tab + (L + 1);        // h at the L nodes
    {
        const int gt = blockIdx.x * kThreads + threadIdx.x, nt = gridDim.x * kThreads;
        for (int e = gt; e <= L; e += nt) tab[e] = cospi((double)e / (2.0 * L));
        for (int l = gt; l < L; l += nt) {
            // cos theta_l = cos(pi (2l + 1) / 2L): m = 2l + 1 <= 2L - 1
            const int m = 2 * l + 1;
            const double c = m > L ? -cospi((double)(2 * L - m) / (2.0 * L)) : cospi((double)m / (2.0 * L));
            hs[l] = response(sp, 0.5 * lam * (c + 1.0));
        }
    }
    lgrid_barrier(bar, target, err, wait);
    double *ts = reinterpret_cast<double *>(lsm);   // tab and hs staged per block
    for (int i = threadIdx.x; i < 2 * L + 1; i += kThreads) ts[i] = __ldcg(tab + i);
    __syncthreads();
    const double *tsh = ts + (L + 1);
    for (int k = gwarp; k < rule.L_max; k += nwarps) {
        if (k >= L) {
            if (lane == 0) coef[k] = 0.0;
            continue;
        }
        const int M4 = 4 * L;
        double a = 0.0;
        for (int l = lane; l < L; l += 32) {
            int mm = (int)(((int64_t)k * (2 * l + 1)) % M4);
            if (mm > 2 * L) mm = M4 - mm;
            a += (mm > L ? -ts[2 * L - mm] : ts[mm]) * tsh[l];
        }
        a = warp_sum_d(a);
        if (lane == 0) coef[k] = 2.0 / (double)L * a;
    }
}

}  // namespace

size_t learn_scratch_doubles(int L_max) { return (size_t)kSlots + 2 * (size_t)L_max + 8; }

cudaError_t learn_bound(const float *G, int64_t ldg, int p, int q, const ShrinkParams &sp, const float *P,
                        double L_scale, double margin, int L_min, int L_max, int L_fallback, int use_lambda,
                        int feat_only, int iters, float *v0, float *v1, float *u0, float *u1, double *acc,
                        double *tabg, unsigned int *bar, int *err, double *out, int *L_out, float *feat,
                        double *theta_out, double *coef, cudaStream_t st, int num_sms, const WaitPolicy &wp) {
    cudaError_t r = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
    if (r != cudaSuccess) return r;
    r = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (r != cudaSuccess) return r;
    int grid = std::min(num_sms, (p + kWarps - 1) / kWarps);
    if (grid < 1) grid = 1;
    const int p4 = (p + 3) & ~3;
    size_t smem = (size_t)p4 * sizeof(float) <= 96 * 1024 ? (size_t)p4 * sizeof(float) : 0;
    if (!feat_only) smem = std::max(smem, (size_t)(2 * L_max + 1) * sizeof(double));
    if (smem > 48 * 1024) {
        r = ensure_smem_limit((const void *)learn_bound_kernel, 160 * 1024);
        if (r != cudaSuccess) return r;
    }
    LearnRule rule{P, L_scale, margin, L_min, L_max, L_fallback, use_lambda, feat_only};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, learn_bound_kernel, G, ldg, p, q, sp, rule, iters, v0, v1, u0, u1, acc, bar, err,
                              out, L_out, feat, theta_out, coef, tabg, wait_limit(wp), wp.stall);
}

}  // namespace cpa
