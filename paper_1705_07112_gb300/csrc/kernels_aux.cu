// Bandwidth-bound helper kernels of the CPA path: the Lambda_max power
// iteration, the device-side Chebyshev coefficients, the shift
// B_hat = (2/Lambda_max) G - Id with the initial sum, and FP32 -> BF16 hi/lo
// splitting of tensor-core operands.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cpa {

cudaError_t ensure_smem_limit(const void *func, int bytes) {
    struct Entry {
        int dev;
        const void *func;
        int bytes;
    };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r != cudaSuccess) return r;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry &e : done)
        if (e.dev == dev && e.func == func && e.bytes >= bytes) return cudaSuccess;
    r = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (r != cudaSuccess) return r;
    for (Entry &e : done)
        if (e.dev == dev && e.func == func) {
            e.bytes = bytes;
            return cudaSuccess;
        }
    done.push_back(Entry{dev, func, bytes});
    return cudaSuccess;
}

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum; blockDim.x a multiple of 32, <= 1024.
__device__ double block_sum(double v) {
    __shared__ double red[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double r = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum(r);
    return r;   // valid in thread 0
}

// SplitMix64 (Steele, Lea, Flood 2014), output i of the generator seeded with
// `seed`: the state after i+1 golden-ratio increments through the finaliser.
__device__ __forceinline__ uint64_t splitmix64_output(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// v0 and |v0|^2; clears the norm slots used by the iteration.
__global__ void power_init_kernel(float *v, int p, uint64_t seed, double *norm2, int nslots) {
    double s = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        uint64_t z = splitmix64_output(seed, (uint64_t)i);
        float x = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
        v[i] = x;
        s += (double)x * (double)x;
    }
    for (int i = threadIdx.x + 1; i < nslots; i += blockDim.x) norm2[i] = 0.0;
    s = block_sum(s);
    if (threadIdx.x == 0) norm2[0] = s;
}

// w = G (v / sqrt(norm_in)),  norm_out += |w|^2.  One warp per row of G.
__global__ void power_matvec_kernel(const float *__restrict__ G, int64_t ldg, int p,
                                    const float *__restrict__ v, const double *norm_in,
                                    float *__restrict__ w, double *norm_out) {
    double nin = *norm_in;
    float scale = nin > 0.0 ? (float)(1.0 / sqrt(nin)) : 0.f;
    int lane = threadIdx.x & 31;
    int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    double contrib = 0.0;
    if (row < p) {
        const float *g = G + (int64_t)row * ldg;
        float s = 0.f;
        if ((ldg & 3) == 0 && (p & 3) == 0 && ((uintptr_t)G & 15) == 0 && ((uintptr_t)v & 15) == 0) {
            const float4 *g4 = reinterpret_cast<const float4 *>(g);
            const float4 *v4 = reinterpret_cast<const float4 *>(v);
            for (int j = lane; j < (p >> 2); j += 32) {
                float4 a = __ldg(g4 + j), b = __ldg(v4 + j);
                s = fmaf(a.x, b.x, s); s = fmaf(a.y, b.y, s);
                s = fmaf(a.z, b.z, s); s = fmaf(a.w, b.w, s);
            }
        } else {
            for (int j = lane; j < p; j += 32) s = fmaf(g[j], v[j], s);
        }
        s = warp_sumf(s) * scale;
        if (lane == 0) {
            w[row] = s;
            contrib = (double)s * (double)s;
        }
    }
    double tot = block_sum(contrib);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(norm_out, tot);
}

// theta = v.w, r = |w - theta v|, trace, lambda (FP64).  v = vu / sqrt(nv).
__global__ void power_final_kernel(const float *vu, const double *nv, const float *w, const double *nw,
                                   const float *G, int64_t ldg, int p, double margin, double *out) {
    double n = *nv;
    double sc = n > 0.0 ? 1.0 / sqrt(n) : 0.0;
    double th = 0.0, tr = 0.0;
    int nonfinite = 0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        th += (double)vu[i] * sc * (double)w[i];
        double gii = (double)G[(int64_t)i * ldg + i];
        tr += gii;
        if (!isfinite(gii)) nonfinite = 1;
    }
    th = block_sum(th);
    __shared__ double sh_th;
    if (threadIdx.x == 0) sh_th = th;
    __syncthreads();
    th = sh_th;
    double r2 = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double d = (double)w[i] - th * (double)vu[i] * sc;
        r2 += d * d;
    }
    r2 = block_sum(r2);
    tr = block_sum(tr);
    nonfinite = __syncthreads_or(nonfinite);
    if (threadIdx.x == 0) {
        double r = sqrt(r2);
        double lam = (th + r) * (1.0 + margin);
        if (lam > tr) lam = tr;
        double flag = 0.0;
        if (nonfinite || !isfinite(lam) || !isfinite(tr)) {
            flag = (double)CPA_ERR_NONFINITE;
        } else if (!(lam > 0.0)) {
            // theta + r = 0 only when X = 0 (trace 0) or v0 lies in the null
            // space; the trace is then the bound, and any positive value
            // serves for X = 0, whose shrinkage is 0.
            lam = tr > 0.0 ? tr : 1.0;
        }
        out[0] = th;
        out[1] = r;
        out[2] = tr;
        out[3] = lam;
        out[4] = flag;
    }
    (void)nw;
}

// Shifted Chebyshev coefficients (Eq. chebychev_coeff_shifted), FP64:
//   c_k = (2/L) sum_l cos(k theta_l) h(lam/2 (cos theta_l + 1)),
//   theta_l = pi (l - 1/2) / L.
// k theta_l = pi k (2l - 1) / (2L), so every cosine is cos(pi m / (2L)) for
// an integer m taken mod 4L: one table of 4L values replaces L^2 cosines
// (FP64 transcendental throughput is low on this part).
__global__ void coeffs_kernel(const double *lam_dev, double lam_host, int L, ShrinkParams s, double *c) {
    extern __shared__ double sh[];
    double *tab = sh;            // [4L]
    double *hs = sh + 4 * L;     // [L]
    const double lam = lam_dev ? lam_dev[0] : lam_host;
    for (int m = threadIdx.x; m < 4 * L; m += blockDim.x) tab[m] = cospi((double)m / (2.0 * L));
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        // cos theta_l = cos(pi (2l+1) / (2L)) for the 0-based l
        const double x = 0.5 * lam * (tab[(2 * l + 1) % (4 * L)] + 1.0);
        hs[l] = response(s, x);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < L; k += nw) {
        double acc = 0.0;
        for (int l = lane; l < L; l += 32) {
            const int m = (int)(((int64_t)k * (2 * l + 1)) % (4 * L));
            acc += tab[m] * hs[l];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) c[k] = 2.0 / (double)L * acc;
    }
}

__device__ __forceinline__ void put_split(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t idx, float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    if (lo) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// B_hat = (2/lambda) G - Id;  Z1 = B_hat;  H = c0/2 Id + c1 B_hat  (the
// initial sum of Algorithm 1).  The product operand is At = (2/lambda) G
// without the -Id, which the recurrence's epilogue applies exactly: FP32 in
// A (CUDA-core path), BF16 hi/lo (tensor-core path); Z1 also as BF16 hi/lo.
// Clenshaw's sum (L >= 3): Z1 = b_{L-2} = c_{L-2} Id + 2 c_{L-1} A instead.
__global__ void shift_kernel(const float *__restrict__ G, int64_t ldg, int p, const double *lam,
                             const double *c, int L, float *A, float *Z1, float *H, int64_t ld,
                             __nv_bfloat16 *Athi, __nv_bfloat16 *Atlo, __nv_bfloat16 *Z1hi, __nv_bfloat16 *Z1lo,
                             int64_t ldb, int clenshaw, __nv_bfloat16 *Z0hi, __nv_bfloat16 *Z0lo, double span,
                             float sigma) {
    // the scalars once per block: an FP64 division in every thread would
    // queue hundreds of thousands of them on this part's scarce FP64 pipe
    __shared__ float sc[5];
    const bool cl = clenshaw && L >= 3;
    if (threadIdx.x == 0) {
        sc[0] = (float)(2.0 / (span > 0.0 ? span : lam[0]));
        sc[1] = (float)(0.5 * c[0]);
        sc[2] = L > 1 ? (float)c[1] : 0.f;
        sc[3] = cl ? (float)c[L - 2] : 0.f;
        sc[4] = cl ? (float)(2.0 * c[L - 1]) : 1.f;
    }
    __syncthreads();
    const float s = sc[0], c0h = sc[1], c1 = sc[2], zc = sc[3], za = sc[4];
    // a block per row (grid-stride), threads across the row: no 64-bit
    // division per element
    for (int i = blockIdx.x; i < p; i += gridDim.x)
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        float at = s * G[(int64_t)i * ldg + j];
        float a = at - (i == j ? sigma : 0.f);
        const float z1 = za * a + (i == j ? zc : 0.f);
        if (A) A[(int64_t)i * ld + j] = at;
        if (Z1) Z1[(int64_t)i * ld + j] = z1;
        H[(int64_t)i * ld + j] = c1 * a + (i == j ? c0h : 0.f);
        if (Athi) put_split(Athi, Atlo, (int64_t)i * ldb + j, at);
        if (Z1hi) put_split(Z1hi, Z1lo, (int64_t)i * ldb + j, z1);
    }
    // zero padding of the BF16 operands' rows (read as contraction columns)
    if (Athi) {
        const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
        for (int i = blockIdx.x; i < p; i += gridDim.x)
            for (int64_t j = p + threadIdx.x; j < ldb; j += blockDim.x) {
                const int64_t o = (int64_t)i * ldb + j;
                Athi[o] = z;
                if (Atlo) Atlo[o] = z;
                if (Z1hi) Z1hi[o] = z;
                if (Z1lo) Z1lo[o] = z;
                if (Z0hi) Z0hi[o] = z;
                if (Z0lo) Z0lo[o] = z;
            }
    }
}

// hi/lo split of a row-major FP32 matrix, optionally transposed, through a
// 32 x 32 shared-memory tile so both the read and the write are coalesced.
__global__ void split_kernel(const float *__restrict__ X, int rows, int cols, int64_t ldx, int transpose,
                             __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ldo) {
    __shared__ float t[32][33];
    int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        int r = r0 + k, c = c0 + tx;
        t[k][tx] = (r < rows && c < cols) ? X[(int64_t)r * ldx + c] : 0.f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        if (!transpose) {
            int r = r0 + k, c = c0 + tx;
            if (r < rows && c < cols) put_split(hi, lo, (int64_t)r * ldo + c, t[k][tx]);
        } else {
            int r = c0 + k, c = r0 + tx;   // out is cols x rows
            if (r < cols && c < rows) put_split(hi, lo, (int64_t)r * ldo + c, t[tx][k]);
        }
    }
}

// hi/lo split of a symmetric matrix stored in its lower triangle (row >= col
// valid): writes both triangles.  Block (bx, by) with by >= bx handles the
// 32 x 32 tile (by, bx) and its transpose through shared memory.
__global__ void split_sym_lower_kernel(const float *__restrict__ S, int p, int64_t lds, __nv_bfloat16 *hi,
                                       __nv_bfloat16 *lo, int64_t ldo) {
    __shared__ float t[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;
    if (by < bx) return;
    const int r0 = by * 32, c0 = bx * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        int r = r0 + k, c = c0 + tx;
        // diagonal tile: take the lower element for both positions
        float v = 0.f;
        if (r < p && c < p) v = (r >= c) ? S[(int64_t)r * lds + c] : S[(int64_t)c * lds + r];
        t[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        int r = r0 + k, c = c0 + tx;
        if (r < p && c < p) put_split(hi, lo, (int64_t)r * ldo + c, t[k][tx]);
        int rt = c0 + k, ct = r0 + tx;   // transposed tile
        if (by != bx && rt < p && ct < p) put_split(hi, lo, (int64_t)rt * ldo + ct, t[tx][k]);
    }
}

__global__ void check_finite_kernel(const float *X, int64_t rows, int64_t cols, int64_t ldx, int *flag) {
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        float v = X[(e / cols) * ldx + e % cols];
        if (!isfinite(v)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// Software grid barrier for a cooperative launch: a monotone arrival
// counter (zeroed before the launch); each block's thread 0 adds one and
// waits for the count of the current round.  The wait is bounded (`limit`
// clock cycles); on expiry it records CPA_ERR_TIMEOUT in *err and lets the
// block go on.  extra: arrivals expected beyond the grid's own (a stalled
// barrier for tests of the timeout path).
__device__ __forceinline__ void grid_barrier(unsigned int *count, unsigned int &target, int *err, long long limit,
                                             unsigned int extra = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x + extra;
        // release: this block's prior writes (made visible to the thread by
        // the CTA barrier) are ordered before the arrival
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

// All power iterations in one cooperative launch.  Iteration t: w_{t+1} =
// G (w_t / |w_t|), one warp per row, |w_{t+1}|^2 summed in FP32 per block and
// in FP64 across blocks (atomics into norm2[t+1]); a grid barrier separates
// iterations; the scale 1/|w_t| is formed in FP32.  Block 0
// then forms theta, r, the trace and lambda as power_final_kernel does.
// Dynamic shared memory: when `cache`, every warp owns at most one row of
// G and keeps it for all iterations (row stride p rounded up to 4); when
// `stage`, the block copies the current iterate once per iteration
// (coalesced 16-byte loads) instead of every warp reading it from L2.
__global__ void __launch_bounds__(512) power_persistent_kernel(const float *__restrict__ G, int64_t ldg, int p,
                                                               int iters, uint64_t seed, float *v0, float *v1,
                                                               double *norm2, unsigned int *bar, double margin,
                                                               double *out, int *err, int cache, int stage,
                                                               int L, ShrinkParams sp, double *coef,
                                                               long long wait_cycles, int stall,
                                                               const int *__restrict__ start_idx) {
    extern __shared__ __align__(16) float grow[];
    __shared__ float wpart[16];    // per-warp |w|^2 partials
    __shared__ float sscale;       // 1 / |v| of the current iterate
    unsigned int target = 0;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    // start vector and its norm (block 0), slots cleared
    if (blockIdx.x == 0) {
        double sacc = 0.0;
        for (int i = p + threadIdx.x; i < ((p + 3) & ~3); i += blockDim.x) {
            v0[i] = 0.f;   // float4 padding of both vectors
            v1[i] = 0.f;
        }
        for (int i = threadIdx.x; i < p; i += blockDim.x) {
            // entry i of the start vector, or entry start_idx[i] of the
            // start vector of the matrix this one is the block of
            uint64_t z = splitmix64_output(seed, (uint64_t)(start_idx ? start_idx[i] : i));
            float x = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
            v0[i] = x;
            sacc += (double)x * (double)x;
        }
        for (int i = threadIdx.x + 1; i < iters + 2; i += blockDim.x) norm2[i] = 0.0;
        sacc = block_sum(sacc);
        if (threadIdx.x == 0) norm2[0] = sacc;
    }
    const int p4 = (p + 3) & ~3;
    float *myrow = grow + (threadIdx.x >> 5) * p4;
    float *vs = grow + (cache ? 16 * p4 : 0);   // staged iterate
    if (cache && gwarp < p) {
        const float *g = G + (int64_t)gwarp * ldg;
        for (int j = lane; j < p4; j += 32) myrow[j] = j < p ? __ldg(g + j) : 0.f;
    }
    grid_barrier(bar, target, err, wait_cycles, stall ? 1u : 0u);
    const bool vec = (ldg & 3) == 0 && (p & 3) == 0 && ((uintptr_t)G & 15) == 0;
    for (int t = 0; t <= iters; ++t) {
        const float *v = (t & 1) ? v1 : v0;
        float *w = (t & 1) ? v0 : v1;
        // 1 / |v| once per block, in FP32 (FP64 square roots and divisions
        // are long dependent sequences on this part's scarce FP64 pipe)
        if (threadIdx.x == 0) {
            const double nin = __ldcg(&norm2[t]);   // written by other blocks: read at L2
            sscale = nin > 0.0 ? __frcp_rn(__fsqrt_rn((float)nin)) : 0.f;
        }
        if (stage) {
            // written by other blocks before the barrier: read at L2
            const float4 *src = reinterpret_cast<const float4 *>(v);
            float4 *dst = reinterpret_cast<float4 *>(vs);
            for (int i = threadIdx.x; i < (p4 >> 2); i += blockDim.x) dst[i] = __ldcg(src + i);
        }
        __syncthreads();
        const float scale = sscale;
        const float *vsrc = stage ? vs : v;
        float part = 0.f;
        for (int row = gwarp; row < p; row += nwarps) {
            const float *g = G + (int64_t)row * ldg;
            float acc = 0.f;
            if (cache) {
                const float4 *g4 = reinterpret_cast<const float4 *>(myrow);
                const float4 *v4 = reinterpret_cast<const float4 *>(vsrc);
                const int n4 = p4 >> 2;
                for (int j0 = lane; j0 < n4; j0 += 32 * 8) {
                    float4 a[8], b[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = j0 + 32 * u;
                        a[u] = j < n4 ? g4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[u] = j < n4 ? (stage ? v4[j] : __ldcg(v4 + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        acc = fmaf(a[u].x, b[u].x, acc); acc = fmaf(a[u].y, b[u].y, acc);
                        acc = fmaf(a[u].z, b[u].z, acc); acc = fmaf(a[u].w, b[u].w, acc);
                    }
                }
            } else if (vec) {
                const float4 *g4 = reinterpret_cast<const float4 *>(g);
                const float4 *v4 = reinterpret_cast<const float4 *>(vsrc);
                const int n4 = p >> 2;
                // eight independent float4 pairs in flight per lane (64 KB a
                // block of 16 warps)
                for (int j0 = lane; j0 < n4; j0 += 32 * 8) {
                    float4 a[8], b[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = j0 + 32 * u;
                        a[u] = j < n4 ? __ldg(g4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[u] = j < n4 ? (stage ? v4[j] : __ldcg(v4 + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        acc = fmaf(a[u].x, b[u].x, acc); acc = fmaf(a[u].y, b[u].y, acc);
                        acc = fmaf(a[u].z, b[u].z, acc); acc = fmaf(a[u].w, b[u].w, acc);
                    }
                }
            } else {
                for (int j = lane; j < p; j += 32) acc = fmaf(__ldg(g + j), stage ? vs[j] : __ldcg(v + j), acc);
            }
            acc = warp_sumf(acc) * scale;
            if (lane == 0) {
                w[row] = acc;
                part = fmaf(acc, acc, part);
            }
        }
        // lane 0 of each warp holds its rows' part (FP32: it only scales
        // the next iterate); one warp adds the 16, one FP64 atomic per block
        if (lane == 0) wpart[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x < 32) {
            float q = threadIdx.x < (int)(blockDim.x >> 5) ? wpart[threadIdx.x] : 0.f;
            q = warp_sumf(q);
            if (threadIdx.x == 0 && q != 0.f) atomicAdd(&norm2[t + 1], (double)q);
        }
        grid_barrier(bar, target, err, wait_cycles);
    }
    // after iters+1 products: v = buffer of step iters (unnormalised, norm2[iters]),
    // w = G v / |v| in the other buffer
    if (blockIdx.x != 0) return;
    const float *vu = (iters & 1) ? v1 : v0;
    const float *w = (iters & 1) ? v0 : v1;
    const double n = __ldcg(&norm2[iters]);
    const double sc = n > 0.0 ? 1.0 / sqrt(n) : 0.0;
    double th = 0.0, tr = 0.0;
    int nonfinite = 0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        th += (double)__ldcg(vu + i) * sc * (double)__ldcg(w + i);
        double gii = (double)G[(int64_t)i * ldg + i];
        tr += gii;
        if (!isfinite(gii)) nonfinite = 1;
    }
    th = block_sum(th);
    __shared__ double sh_th;
    if (threadIdx.x == 0) sh_th = th;
    __syncthreads();
    th = sh_th;
    double r2 = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double d = (double)__ldcg(w + i) - th * (double)__ldcg(vu + i) * sc;
        r2 += d * d;
    }
    r2 = block_sum(r2);
    tr = block_sum(tr);
    nonfinite = __syncthreads_or(nonfinite);
    if (threadIdx.x == 0) {
        double r = sqrt(r2);
        double lam = (th + r) * (1.0 + margin);
        if (lam > tr) lam = tr;
        double flag = 0.0;
        if (nonfinite || !isfinite(lam) || !isfinite(tr)) {
            flag = (double)CPA_ERR_NONFINITE;
        } else if (!(lam > 0.0)) {
            lam = tr > 0.0 ? tr : 1.0;
        }
        const int e2 = __ldcg(err);
        if (e2) flag = (double)e2;
        out[0] = th;
        out[1] = r;
        out[2] = tr;
        out[3] = lam;
        out[4] = flag;
        sh_th = lam;
    }
    if (!coef) return;
    // the coefficients of Eq. chebychev_coeff_shifted on [0, lambda] in the
    // same block (as coeffs_kernel computes them), in the shared memory the
    // rows of G used: table cos(pi m / 2L), m < 4L, then h at the L nodes
    __syncthreads();
    const double lamv = sh_th;
    double *tab = reinterpret_cast<double *>(grow);
    double *hs = tab + 4 * L;
    for (int m = threadIdx.x; m < 4 * L; m += blockDim.x) tab[m] = cospi((double)m / (2.0 * L));
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) hs[l] = response(sp, 0.5 * lamv * (tab[(2 * l + 1) % (4 * L)] + 1.0));
    __syncthreads();
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < L; k += nw) {
        double acc = 0.0;
        for (int l = lane; l < L; l += 32) {
            const int m = (int)(((int64_t)k * (2 * l + 1)) % (4 * L));
            acc += tab[m] * hs[l];
        }
        acc = warp_sum(acc);
        if (lane == 0) coef[k] = 2.0 / (double)L * acc;
    }
}

}  // namespace

cudaError_t power_bound_persistent(const float *G, int64_t ldg, int p, int iters, float *v0, float *v1,
                                   double *norm2, unsigned int *bar, int *err, double *out, cudaStream_t st,
                                   int num_sms, int L, const ShrinkParams *sp, double *coef, const WaitPolicy &wp,
                                   const int *start_idx) {
    cudaError_t r = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
    if (r != cudaSuccess) return r;
    r = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (r != cudaSuccess) return r;
    int grid = num_sms;
    const int rows_per_block = 16;   // warps per block
    if (grid > (p + rows_per_block - 1) / rows_per_block) grid = (p + rows_per_block - 1) / rows_per_block;
    if (grid < 1) grid = 1;
    const int p4 = (p + 3) & ~3;
    const size_t budget = 200 * 1024;
    const size_t cache_bytes = (size_t)16 * p4 * sizeof(float);
    const int cache = ((int64_t)grid * 16 >= p && cache_bytes <= budget) ? 1 : 0;
    const size_t stage_bytes = (size_t)p4 * sizeof(float);
    const int stage = (cache ? cache_bytes : 0) + stage_bytes <= budget ? 1 : 0;
    size_t smem = (cache ? cache_bytes : 0) + (stage ? stage_bytes : 0);
    // the coefficient table and node values reuse the same shared memory
    if (coef && (L < 1 || L > kMaxTerms || !sp)) return cudaErrorInvalidValue;
    if (coef && smem < (size_t)5 * L * sizeof(double)) smem = (size_t)5 * L * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t ra = ensure_smem_limit((const void *)power_persistent_kernel, (int)budget);
        if (ra != cudaSuccess) return ra;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double margin = kLambdaMargin;
    const uint64_t seed = kStartSeed;
    const ShrinkParams spv = sp ? *sp : ShrinkParams{};
    return cudaLaunchKernelEx(&cfg, power_persistent_kernel, G, ldg, p, iters, seed, v0, v1, norm2, bar, margin, out,
                              err, cache, stage, coef ? L : 0, spv, coef, wait_limit(wp), wp.stall, start_idx);
}

cudaError_t power_bound(const float *G, int64_t ldg, int p, int iters, float *v0, float *v1,
                        double *norm2, double *out, cudaStream_t st) {
    power_init_kernel<<<1, 1024, 0, st>>>(v0, p, kStartSeed, norm2, iters + 2);
    float *bufs[2] = {v0, v1};
    int threads = 256;
    int blocks = (int)(((int64_t)p * 32 + threads - 1) / threads);
    for (int t = 0; t < iters; ++t)
        power_matvec_kernel<<<blocks, threads, 0, st>>>(G, ldg, p, bufs[t & 1], norm2 + t, bufs[(t + 1) & 1],
                                                        norm2 + t + 1);
    // final product w = G v with v = bufs[iters&1] / sqrt(norm2[iters])
    float *vu = bufs[iters & 1], *w = bufs[(iters + 1) & 1];
    power_matvec_kernel<<<blocks, threads, 0, st>>>(G, ldg, p, vu, norm2 + iters, w, norm2 + iters + 1);
    // the final kernel needs v unscaled and w: w overwrote the other buffer,
    // vu is intact
    power_final_kernel<<<1, 1024, 0, st>>>(vu, norm2 + iters, w, norm2 + iters + 1, G, ldg, p, kLambdaMargin,
                                           out);
    return cudaGetLastError();
}

cudaError_t device_coeffs(const double *lam_dev, double lam_host, int L, const ShrinkParams &s, double *c,
                          cudaStream_t st) {
    const size_t smem = (size_t)5 * L * sizeof(double);
    cudaError_t r = ensure_smem_limit((const void *)coeffs_kernel, 5 * kMaxTerms * (int)sizeof(double));
    if (r != cudaSuccess) return r;
    coeffs_kernel<<<1, 1024, smem, st>>>(lam_dev, lam_host, L, s, c);
    return cudaGetLastError();
}

// H = (b_0 - b_2) / 2, b_0 in H, b_2 in B2 or c[2] Id.
__global__ void clenshaw_finish_kernel(float *H, const float *B2, int p, int64_t ld, const double *c,
                                       int lower_only) {
    const float c2 = B2 ? 0.f : (float)c[2];
    for (int i = blockIdx.x; i < p; i += gridDim.x)
        for (int j = threadIdx.x; j <= (lower_only ? i : p - 1); j += blockDim.x) {
            const int64_t o = (int64_t)i * ld + j;
            const float b2 = (B2 ? B2[o] : 0.f) + (i == j ? c2 : 0.f);
            H[o] = 0.5f * (H[o] - b2);
        }
}

cudaError_t shift_init(const float *G, int64_t ldg, int p, const double *lam, const double *c, int L, float *A,
                       float *Z1, float *H, int64_t ld, __nv_bfloat16 *Athi, __nv_bfloat16 *Atlo,
                       __nv_bfloat16 *Z1hi, __nv_bfloat16 *Z1lo, int64_t ldb, cudaStream_t st, int num_sms,
                       int clenshaw, __nv_bfloat16 *Z0hi, __nv_bfloat16 *Z0lo, double span, double sigma) {
    int blocks = std::min(p, num_sms * 8);   // a block per row, grid-stride
    if (blocks < 1) blocks = 1;
    shift_kernel<<<blocks, 256, 0, st>>>(G, ldg, p, lam, c, L, A, Z1, H, ld, Athi, Atlo, Z1hi, Z1lo, ldb,
                                         clenshaw, Z0hi, Z0lo, span, (float)sigma);
    return cudaGetLastError();
}

void coeffs_interval(const ShrinkParams &s, int L, double a, double b, double *c) {
    for (int k = 0; k < L; ++k) {
        double acc = 0.0;
        for (int l = 1; l <= L; ++l) {
            const double th = kPi * ((double)l - 0.5) / (double)L;
            const double x = a + 0.5 * (b - a) * (cos(th) + 1.0);
            acc += cos((double)k * th) * (x > 0.0 ? response(s, x) : 0.0);
        }
        c[k] = 2.0 / (double)L * acc;
    }
}

cudaError_t split_bf16(const float *X, int rows, int cols, int64_t ldx, bool transpose, __nv_bfloat16 *hi,
                       __nv_bfloat16 *lo, int64_t ldo, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    split_kernel<<<grid, dim3(32, 8), 0, st>>>(X, rows, cols, ldx, transpose ? 1 : 0, hi, lo, ldo);
    return cudaGetLastError();
}

cudaError_t split_sym_lower(const float *S, int p, int64_t lds, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ldo,
                            cudaStream_t st) {
    dim3 grid((p + 31) / 32, (p + 31) / 32);
    split_sym_lower_kernel<<<grid, dim3(32, 8), 0, st>>>(S, p, lds, hi, lo, ldo);
    return cudaGetLastError();
}

cudaError_t check_finite(const float *X, int64_t rows, int64_t cols, int64_t ldx, int *flag, cudaStream_t st,
                         int num_sms) {
    int64_t total = rows * cols;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<blocks, 256, 0, st>>>(X, rows, cols, ldx, flag);
    return cudaGetLastError();
}

cudaError_t clenshaw_finish(float *H, const float *B2, int p, int64_t ld, const double *c, int lower_only,
                            cudaStream_t st, int num_sms) {
    int blocks = std::min(p, num_sms * 8);
    if (blocks < 1) blocks = 1;
    clenshaw_finish_kernel<<<blocks, 256, 0, st>>>(H, B2, p, ld, c, lower_only);
    return cudaGetLastError();
}

}  // namespace cpa
