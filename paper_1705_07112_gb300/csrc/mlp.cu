// Small fully connected network for the learned Lambda_max / order
// predictor: in -> h1 -> h2 -> out, ReLU on the hidden layers, FP32.
// Forward, backward (loss = (1/2B) sum_b sum_o (y_bo - t_bo)^2) and Adam run
// in the kernels below; the paper has no counterpart (the predictor is a
// deployment aid that chooses Lambda_max and L for Algorithm 1).
//
// Parameter layout (one contiguous FP32 array):
//   W1 [h1][in], b1 [h1], W2 [h2][h1], b2 [h2], W3 [out][h2], b3 [out].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace cpa {
namespace {

constexpr int kMaxWidth = 128;

struct Dims {
    int in, h1, h2, out;
    int oW1, ob1, oW2, ob2, oW3, ob3, total;
};

Dims make_dims(int in, int h1, int h2, int out) {
    Dims d{in, h1, h2, out, 0, 0, 0, 0, 0, 0, 0};
    d.oW1 = 0;
    d.ob1 = d.oW1 + h1 * in;
    d.oW2 = d.ob1 + h1;
    d.ob2 = d.oW2 + h2 * h1;
    d.oW3 = d.ob2 + h2;
    d.ob3 = d.oW3 + out * h2;
    d.total = d.ob3 + out;
    return d;
}

// One thread per sample: forward pass; optionally keeps the hidden
// activations (for backward) in act[b][h1 + h2].
__global__ void mlp_forward_kernel(Dims d, const float *__restrict__ P, const float *__restrict__ X, int batch,
                                   float *__restrict__ Y, float *__restrict__ act) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    float h1[kMaxWidth], h2[kMaxWidth];
    const float *x = X + (int64_t)b * d.in;
    for (int i = 0; i < d.h1; ++i) {
        float s = P[d.ob1 + i];
        for (int j = 0; j < d.in; ++j) s = fmaf(P[d.oW1 + i * d.in + j], x[j], s);
        h1[i] = s > 0.f ? s : 0.f;
    }
    for (int i = 0; i < d.h2; ++i) {
        float s = P[d.ob2 + i];
        for (int j = 0; j < d.h1; ++j) s = fmaf(P[d.oW2 + i * d.h1 + j], h1[j], s);
        h2[i] = s > 0.f ? s : 0.f;
    }
    for (int i = 0; i < d.out; ++i) {
        float s = P[d.ob3 + i];
        for (int j = 0; j < d.h2; ++j) s = fmaf(P[d.oW3 + i * d.h2 + j], h2[j], s);
        Y[(int64_t)b * d.out + i] = s;
    }
    if (act) {
        float *a = act + (int64_t)b * (d.h1 + d.h2);
        for (int i = 0; i < d.h1; ++i) a[i] = h1[i];
        for (int i = 0; i < d.h2; ++i) a[d.h1 + i] = h2[i];
    }
}

// Backward: gradients of the loss summed over the batch into G (zeroed
// first), one thread per sample, block partial sums in shared memory, one
// atomic per parameter per block.  loss (device scalar) accumulates the
// loss value.
__global__ void mlp_backward_kernel(Dims d, const float *__restrict__ P, const float *__restrict__ X,
                                    const float *__restrict__ Y, const float *__restrict__ T,
                                    const float *__restrict__ act, int batch, float *__restrict__ G,
                                    float *__restrict__ loss) {
    extern __shared__ float gs[];   // [d.total]
    for (int i = threadIdx.x; i < d.total; i += blockDim.x) gs[i] = 0.f;
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const float inv = 1.f / (float)batch;
    float my_loss = 0.f;
    if (b < batch) {
        const float *x = X + (int64_t)b * d.in;
        const float *h1 = act + (int64_t)b * (d.h1 + d.h2);
        const float *h2 = h1 + d.h1;
        float dy[kMaxWidth], dh2[kMaxWidth], dh1[kMaxWidth];
        for (int o = 0; o < d.out; ++o) {
            const float r = Y[(int64_t)b * d.out + o] - T[(int64_t)b * d.out + o];
            my_loss += 0.5f * r * r * inv;
            dy[o] = r * inv;
        }
        for (int j = 0; j < d.h2; ++j) dh2[j] = 0.f;
        for (int o = 0; o < d.out; ++o) {
            atomicAdd(&gs[d.ob3 + o], dy[o]);
            for (int j = 0; j < d.h2; ++j) {
                atomicAdd(&gs[d.oW3 + o * d.h2 + j], dy[o] * h2[j]);
                dh2[j] = fmaf(P[d.oW3 + o * d.h2 + j], dy[o], dh2[j]);
            }
        }
        for (int j = 0; j < d.h2; ++j) dh2[j] = h2[j] > 0.f ? dh2[j] : 0.f;
        for (int j = 0; j < d.h1; ++j) dh1[j] = 0.f;
        for (int i = 0; i < d.h2; ++i) {
            if (dh2[i] == 0.f) continue;
            atomicAdd(&gs[d.ob2 + i], dh2[i]);
            for (int j = 0; j < d.h1; ++j) {
                atomicAdd(&gs[d.oW2 + i * d.h1 + j], dh2[i] * h1[j]);
                dh1[j] = fmaf(P[d.oW2 + i * d.h1 + j], dh2[i], dh1[j]);
            }
        }
        for (int i = 0; i < d.h1; ++i) {
            const float g = h1[i] > 0.f ? dh1[i] : 0.f;
            if (g == 0.f) continue;
            atomicAdd(&gs[d.ob1 + i], g);
            for (int j = 0; j < d.in; ++j) atomicAdd(&gs[d.oW1 + i * d.in + j], g * x[j]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
    if ((threadIdx.x & 31) == 0 && my_loss != 0.f && loss) atomicAdd(loss, my_loss);
    __syncthreads();
    for (int i = threadIdx.x; i < d.total; i += blockDim.x)
        if (gs[i] != 0.f) atomicAdd(&G[i], gs[i]);
}

// Adam (Kingma and Ba, 2015) with bias correction, step t counting from 1,
// and decoupled weight decay wd (Loshchilov and Hutter, 2019):
//   P <- P - lr (m_hat / (sqrt(v_hat) + eps) + wd P).
__global__ void adam_kernel(float *P, const float *G, float *M, float *V, int n, float lr, float wd, float b1,
                            float b2, float eps, int t) {
    const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * ((m * c1) / (sqrtf(v * c2) + eps) + wd * P[i]);
    }
}

}  // namespace
}  // namespace cpa

using namespace cpa;

struct cpa_mlp_ctx {
    Dims d;
    int device = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr, *loss = nullptr;
    float *act = nullptr, *Y = nullptr;
    int cap = 0;   // batch capacity of act / Y
    int t = 0;     // Adam step
};

namespace cpa {
const float *mlp_device_params(cpa_mlp m, int dims[4], int *device) {
    if (!m) return nullptr;
    dims[0] = m->d.in;
    dims[1] = m->d.h1;
    dims[2] = m->d.h2;
    dims[3] = m->d.out;
    *device = m->device;
    return m->P;
}
}  // namespace cpa

namespace {

cpa_status mlp_cuda(cudaError_t e) { return e == cudaSuccess ? CPA_OK : CPA_ERR_CUDA; }

cpa_status mlp_reserve(cpa_mlp_ctx *m, int batch, cudaStream_t st) {
    if (batch <= m->cap) return CPA_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CPA_ERR_CUDA;
    cudaFree(m->act);
    cudaFree(m->Y);
    m->act = m->Y = nullptr;
    if (cudaMalloc(&m->act, sizeof(float) * (size_t)batch * (m->d.h1 + m->d.h2)) != cudaSuccess ||
        cudaMalloc(&m->Y, sizeof(float) * (size_t)batch * m->d.out) != cudaSuccess)
        return CPA_ERR_NO_MEMORY;
    m->cap = batch;
    return CPA_OK;
}

}  // namespace

extern "C" {

cpa_status cpa_mlp_create(cpa_mlp *out, int in, int h1, int h2, int outdim, uint64_t seed) {
    if (!out || in < 1 || h1 < 1 || h2 < 1 || outdim < 1 || in > kMaxWidth || h1 > kMaxWidth || h2 > kMaxWidth ||
        outdim > kMaxWidth)
        return CPA_ERR_INVALID_ARG;
    *out = nullptr;
    cpa_mlp m = new cpa_mlp_ctx();
    m->d = make_dims(in, h1, h2, outdim);
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return CPA_ERR_CUDA;
    }
    const size_t bytes = sizeof(float) * m->d.total;
    if (cudaMalloc(&m->P, bytes) != cudaSuccess || cudaMalloc(&m->G, bytes) != cudaSuccess ||
        cudaMalloc(&m->M, bytes) != cudaSuccess || cudaMalloc(&m->V, bytes) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
        cpa_mlp_destroy(m);
        return CPA_ERR_NO_MEMORY;
    }
    // He-style initialisation from a SplitMix64 stream (uniform, variance 2/fan_in)
    std::vector<float> p(m->d.total, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ULL;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int count, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < count; ++i) p[off + i] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(m->d.oW1, m->d.h1 * in, in);
    fill(m->d.oW2, m->d.h2 * h1, h1);
    fill(m->d.oW3, outdim * h2, h2);
    if (cudaMemcpy(m->P, p.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M, 0, bytes) != cudaSuccess || cudaMemset(m->V, 0, bytes) != cudaSuccess) {
        cpa_mlp_destroy(m);
        return CPA_ERR_CUDA;
    }
    *out = m;
    return CPA_OK;
}

cpa_status cpa_mlp_destroy(cpa_mlp m) {
    if (!m) return CPA_ERR_INVALID_ARG;
    cudaFree(m->P);
    cudaFree(m->G);
    cudaFree(m->M);
    cudaFree(m->V);
    cudaFree(m->loss);
    cudaFree(m->act);
    cudaFree(m->Y);
    delete m;
    return CPA_OK;
}

int64_t cpa_mlp_param_count(cpa_mlp m) { return m ? m->d.total : -1; }

cpa_status cpa_mlp_set_params(cpa_mlp m, const float *host, int64_t count) {
    if (!m || !host || count != m->d.total) return CPA_ERR_INVALID_ARG;
    if (cudaMemcpy(m->P, host, sizeof(float) * count, cudaMemcpyHostToDevice) != cudaSuccess) return CPA_ERR_CUDA;
    m->t = 0;
    cudaMemset(m->M, 0, sizeof(float) * count);
    cudaMemset(m->V, 0, sizeof(float) * count);
    return CPA_OK;
}

cpa_status cpa_mlp_get_params(cpa_mlp m, float *host, int64_t count) {
    if (!m || !host || count != m->d.total) return CPA_ERR_INVALID_ARG;
    return mlp_cuda(cudaMemcpy(host, m->P, sizeof(float) * count, cudaMemcpyDeviceToHost));
}

cpa_status cpa_mlp_forward(cpa_mlp m, const float *dX, int batch, float *dY, void *stream) {
    if (!m || !dX || !dY || batch < 0) return CPA_ERR_INVALID_ARG;
    if (batch == 0) return CPA_OK;
    mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->d, m->P, dX, batch, dY, nullptr);
    return mlp_cuda(cudaGetLastError());
}

cpa_status cpa_mlp_gradients(cpa_mlp m, const float *dX, const float *dT, int batch, float *host_grad,
                             int64_t count, float *host_loss, void *stream) {
    if (!m || !dX || !dT || batch < 1 || (host_grad && count != m->d.total)) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cpa_status s = mlp_reserve(m, batch, st);
    if (s != CPA_OK) return s;
    if (cudaMemsetAsync(m->G, 0, sizeof(float) * m->d.total, st) != cudaSuccess ||
        cudaMemsetAsync(m->loss, 0, sizeof(float), st) != cudaSuccess)
        return CPA_ERR_CUDA;
    mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, st>>>(m->d, m->P, dX, batch, m->Y, m->act);
    mlp_backward_kernel<<<(batch + 127) / 128, 128, sizeof(float) * m->d.total, st>>>(m->d, m->P, dX, m->Y, dT,
                                                                                     m->act, batch, m->G, m->loss);
    if (cudaGetLastError() != cudaSuccess) return CPA_ERR_CUDA;
    if (host_grad &&
        cudaMemcpyAsync(host_grad, m->G, sizeof(float) * m->d.total, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CPA_ERR_CUDA;
    if (host_loss && cudaMemcpyAsync(host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CPA_ERR_CUDA;
    return mlp_cuda(cudaStreamSynchronize(st));
}

cpa_status cpa_mlp_train_step(cpa_mlp m, const float *dX, const float *dT, int batch, float lr,
                              float weight_decay, float *host_loss, void *stream) {
    if (!m || !dX || !dT || batch < 1 || !(lr > 0.f) || !(weight_decay >= 0.f)) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cpa_status s = mlp_reserve(m, batch, st);
    if (s != CPA_OK) return s;
    if (cudaMemsetAsync(m->G, 0, sizeof(float) * m->d.total, st) != cudaSuccess ||
        cudaMemsetAsync(m->loss, 0, sizeof(float), st) != cudaSuccess)
        return CPA_ERR_CUDA;
    mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, st>>>(m->d, m->P, dX, batch, m->Y, m->act);
    mlp_backward_kernel<<<(batch + 127) / 128, 128, sizeof(float) * m->d.total, st>>>(m->d, m->P, dX, m->Y, dT,
                                                                                     m->act, batch, m->G, m->loss);
    m->t += 1;
    adam_kernel<<<std::max(1, std::min(1024, (m->d.total + 255) / 256)), 256, 0, st>>>(
        m->P, m->G, m->M, m->V, m->d.total, lr, weight_decay, 0.9f, 0.999f, 1e-8f, m->t);
    if (cudaGetLastError() != cudaSuccess) return CPA_ERR_CUDA;
    if (host_loss) {
        if (cudaMemcpyAsync(host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return CPA_ERR_CUDA;
        return mlp_cuda(cudaStreamSynchronize(st));
    }
    return CPA_OK;
}

}  // extern "C"
