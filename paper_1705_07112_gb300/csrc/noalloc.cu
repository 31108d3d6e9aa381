// Allocation-free variant of the Lambda_max bound.
//
// Some callers cannot allocate device memory when they need the bound:
// latency-critical loops that cannot afford the device-wide synchronisation
// that cudaMalloc/cudaFree imply, services that run under a fixed device
// memory budget which must not grow after start-up, and processes whose
// device memory is already handed out by another allocator (a framework's
// caching pool), where one more cudaMalloc fails or fragments that pool.
// For them this entry point
// computes the same bound as cpa_lambda_bound without a handle and without
// allocating: its scratch (the Gram matrix, the two iteration vectors, the
// FP64 norm slots and the grid-barrier words) lives in one fixed array in
// device global memory, defined below, which every GPU that loads the
// library holds until the process exits.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoAllocMaxP = 512;          // largest min(m, n)
constexpr int kNoAllocMaxIters = 1000;     // largest iteration count
constexpr size_t kNoAllocG = (size_t)kNoAllocMaxP * kNoAllocMaxP;   // floats
constexpr size_t kNoAllocBytes = kNoAllocG * 4 + 2 * kNoAllocMaxP * 4 + (kNoAllocMaxIters + 2) * 8 + 8 * 8 + 256;

// The scratch array (a little over 1 MB per device).  In host code its name
// only stands in for the device object; the device address is obtained with
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current),
// looked up once per device.
cudaError_t scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t r = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (r != cudaSuccess) return r;
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return cudaSuccess;
}

}  // namespace

extern "C" {

cpa_status cpa_lambda_bound_noalloc(const float *dX, int64_t m, int64_t n, int64_t ldx, int iters,
                                    double *lambda_out, void *stream) {
    using namespace cpa;
    if (!dX || !lambda_out || m < 1 || n < 1 || ldx < n || iters < 0 || iters > kNoAllocMaxIters)
        return CPA_ERR_INVALID_ARG;
    const int64_t p = m < n ? m : n;
    if (p > kNoAllocMaxP || (m > n ? m : n) > ((int64_t)1 << 24)) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return CPA_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) return CPA_ERR_CUDA;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return CPA_ERR_CUDA;

    // carve the array: G (p x ldp), v0, v1, norm slots, {theta, r, trace,
    // lambda, status}, barrier counter and error word
    const int64_t ldp = (p + 7) / 8 * 8;
    float *G = reinterpret_cast<float *>(base);
    float *v0 = G + kNoAllocG;
    float *v1 = v0 + kNoAllocMaxP;
    double *norm2 = reinterpret_cast<double *>(v1 + kNoAllocMaxP);
    double *out = norm2 + (kNoAllocMaxIters + 2);
    unsigned int *bar = reinterpret_cast<unsigned int *>(out + 8);
    int *err = reinterpret_cast<int *>(bar + 1);
    if ((size_t)(p * ldp) > kNoAllocG) return CPA_ERR_INVALID_ARG;

    // Gram matrix of the smaller side (every element written; nothing needs
    // clearing).  The power-iteration launcher clears the barrier counter and
    // the error word, and the kernel clears its norm slots, before use.
    Epilogue e;
    e.D = G;
    e.ldd = ldp;
    e.symmetric_upper = 1;
    cudaError_t r;
    if (m >= n)
        r = gemm_f32((int)p, (int)p, (int)m, dX, ldx, false, dX, ldx, false, e, st);
    else
        r = gemm_f32((int)p, (int)p, (int)n, dX, ldx, true, dX, ldx, true, e, st);
    if (r != cudaSuccess) return CPA_ERR_CUDA;
    r = power_bound_persistent(G, ldp, (int)p, iters, v0, v1, norm2, bar, err, out, st, num_sms);
    if (r != cudaSuccess) return CPA_ERR_CUDA;
    double res[5];
    if (cudaMemcpyAsync(res, out, sizeof res, cudaMemcpyDeviceToHost, st) != cudaSuccess) return CPA_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CPA_ERR_CUDA;
    if (res[4] != 0.0) return (cpa_status)(int)res[4];
    *lambda_out = res[3];
    return CPA_OK;
}

}  // extern "C"
