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
#include <algorithm>

#include "internal.h"

namespace cpa {
namespace {

__device__ double dct_entry(int size, int k, int j) {
    const double s = (k == 0) ? sqrt(1.0 / size) : sqrt(2.0 / size);
    return s * cospi((2.0 * j + 1.0) * k / (2.0 * size));
}

__global__ void make_transform_kernel(int type, int p, float *T, int64_t ld) {
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
            v = dct_entry(p, i, j);
        }
        T[(int64_t)i * ld + j] = (float)v;
    }
}

// Entries below eps set to zero; removed2 (optional) accumulates the sum of
// their squares, |Phi - Phi_|_F^2 (per-warp FP32 partials, FP64 atomics).
__global__ void threshold_kernel(float *Phi, int p, int64_t ld, const float *eps_dev, float eps_host,
                                 double *removed2) {
    const float eps = eps_dev ? *eps_dev : eps_host;
    const int64_t total = (int64_t)p * p;
    float r2 = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        float *q = Phi + (e / p) * ld + e % p;
        const float v = *q;
        if (!(fabsf(v) >= eps)) {
            r2 = fmaf(v, v, r2);
            *q = 0.f;
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

// eps = k-th largest |Phi_ij| by a bitwise search over the IEEE bit patterns
// of |Phi| (order-preserving for non-negative floats): bit b from 30 down to
// 0 is kept when at least k entries are >= the candidate.  One cooperative
// launch; a grid barrier per bit.
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

__global__ void topk_eps_kernel(const float *__restrict__ Phi, int p, int64_t ld, long long k,
                                unsigned long long *counts /*[31]*/, unsigned int *bar, int *err, float *eps_out) {
    unsigned int target = 0;
    unsigned int t = 0;
    const int64_t total = (int64_t)p * p;
    for (int bit = 30; bit >= 0; --bit) {
        const unsigned int cand = t | (1u << bit);
        unsigned long long c = 0;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const unsigned int b = __float_as_uint(fabsf(__ldg(Phi + (e / p) * ld + e % p)));
            c += (b >= cand) ? 1ull : 0ull;
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&counts[bit], c);
        grid_sync_sp(bar, target, err);
        if (__ldcg(&counts[bit]) >= (unsigned long long)k) t = cand;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *eps_out = __uint_as_float(t);
}

}  // namespace

cudaError_t make_transform(int type, int p, float *T, int64_t ld, cudaStream_t st, int num_sms) {
    const int64_t total = (int64_t)p * p;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    make_transform_kernel<<<std::max(blocks, 1), 256, 0, st>>>(type, p, T, ld);
    return cudaGetLastError();
}

cudaError_t threshold_entries(float *Phi, int p, int64_t ld, const float *eps_dev, float eps_host, cudaStream_t st,
                              int num_sms, double *removed2) {
    const int64_t total = (int64_t)p * p;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    threshold_kernel<<<std::max(blocks, 1), 256, 0, st>>>(Phi, p, ld, eps_dev, eps_host, removed2);
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
    cudaError_t r = cudaMemsetAsync(counts, 0, 31 * sizeof(unsigned long long), st);
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
