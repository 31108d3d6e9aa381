// C ABI of libcpa: argument checking, workspace management and the launch
// sequence of Algorithm 1 (Gram -> Lambda_max bound -> coefficients -> shift
// -> recurrence with fused accumulation -> final product).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

using namespace cpa;

namespace {
// below this p the BF16 mode also splits the recurrence operands
constexpr int64_t kSplitRecBelow = 256;
constexpr int kMaxStreams = 64;   // concurrent member streams of the pointer-form batches
}  // namespace

struct cpa_ctx {
    int device = 0;
    int num_sms = 0;
    int cc = 0;
    char *ws = nullptr;       // device workspace
    size_t ws_bytes = 0;
    double *h_pin = nullptr;  // pinned host scalars for read-back
    // layout of the last cpa_svt (for the query functions)
    double *d_out = nullptr;  // {theta, r, trace, lambda, status}
    double *d_coef = nullptr;
    int last_L = 0;
    bool have_last = false;
    int series = CPA_SERIES_FORWARD;   // how the filter's series is summed
    WaitPolicy wait;                   // grid-barrier wait limit, test stall
    int *d_err = nullptr;              // error word of the last cpa_svt's tensor-core kernels
    int sparse_skip = 1;               // skip zero tiles of the thresholded operand
    int sparse_compact = 1;            // recurrence on the thresholded operand's nonzero block
    bool have_learn = false;           // the last call chose its order on the device
    int *d_L = nullptr;                // {L, fallback} of that call
    // pointer-form batches (cpa_svt_batched, cpa_serve_learned): the
    // patch-sized members' launch, and per-member choices of the larger
    // members of the last learned call ({L, fallback} pairs, bounds)
    PtrPlan *pplan = nullptr;          // members up to 64 x 128 (mma.sync kernel)
    PtrPlan *pplan_tc = nullptr;       // members up to 128 x 4096 beyond those (tcgen05 kernel)
    std::vector<int> serve_mid;        // member indices of the last learned call in the second group
    int *d_big_L = nullptr;
    double *d_big_lam = nullptr;
    int big_cap = 0;
    std::vector<int> serve_small, serve_big;   // member indices of the last learned call
    // concurrent members: sub-handles (own workspace), each on its own
    // stream forked from the caller's
    int nstreams = 1;
    int member_sms = 0;                // SMs per member on those streams (0: all)
    cpa_ctx *sub[kMaxStreams] = {};
    cudaStream_t sub_st[kMaxStreams] = {};
    cudaEvent_t sub_ev[kMaxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    // diagnostics
    bool profiling = false;
    int64_t launches[CPA_NSTAGES] = {};
    double ms[CPA_NSTAGES] = {};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> event_pool;
    // host-buffer streaming (cpa_svt_host): two device slots of X and Y, one
    // copy stream per direction, slot events
    float *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t in_ready[2] = {}, computed[2] = {}, out_done[2] = {}, start = nullptr;
};

namespace {

cudaEvent_t take_event(cpa_ctx *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one stage (or one launch of a stage) with events when profiling,
// and counts its kernel launches.
struct StageScope {
    cpa_ctx *h;
    int stage;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    StageScope(cpa_ctx *h_, int stage_, cudaStream_t st_, int nlaunch) : h(h_), stage(stage_), st(st_) {
        h->launches[stage] += nlaunch;
        if (h->profiling) {
            e0 = take_event(h);
            cudaEventRecord(e0, st);
        }
    }
    ~StageScope() {
        if (h->profiling && e0) {
            cudaEvent_t e1 = take_event(h);
            cudaEventRecord(e1, st);
            h->pending.push_back({stage, {e0, e1}});
        }
    }
};

}  // namespace

namespace {

thread_local char g_err[256] = "";

cpa_status cuda_fail(cudaError_t e, const char *where) {
    snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
    return CPA_ERR_CUDA;
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

cpa_status check_shrink(const cpa_shrink *s) {
    if (!s) return CPA_ERR_INVALID_ARG;
    if (s->kind == CPA_HARD || s->kind == CPA_SOFT) {
        if (!(s->tau >= 0.0) || !std::isfinite(s->tau)) return CPA_ERR_INVALID_ARG;
    } else if (s->kind == CPA_WSOFT) {
        if (!(s->c >= 0.0) || !(s->eps > 0.0) || !(s->noise >= 0.0) || !std::isfinite(s->c) ||
            !std::isfinite(s->noise))
            return CPA_ERR_INVALID_ARG;
    } else {
        return CPA_ERR_INVALID_ARG;
    }
    return CPA_OK;
}

ShrinkParams to_params(const cpa_shrink *s) {
    ShrinkParams p;
    p.kind = s->kind;
    p.tau = s->tau;
    p.c = s->c;
    p.eps = s->eps;
    p.noise = s->noise;
    return p;
}

// Bump allocator over the handle's workspace; 256-byte aligned pieces.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(char *b) : base(b) {}
    template <class T>
    T *take(size_t count) {
        off = (size_t)round_up((int64_t)off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

cpa_status ensure_ws(cpa_ctx *h, size_t bytes, cudaStream_t st) {
    if (bytes <= h->ws_bytes) return CPA_OK;
    if (h->ws) {
        CK(cudaStreamSynchronize(st));
        CK(cudaDeviceSynchronize());
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = (size_t)round_up((int64_t)bytes, 1 << 20);
    cudaError_t e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        snprintf(g_err, sizeof g_err, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        return CPA_ERR_NO_MEMORY;
    }
    h->ws_bytes = want;
    return CPA_OK;
}

__global__ void set_scalar2_kernel(double *p, double v0, double v1) {
    p[0] = v0;
    p[1] = v1;
}

bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
    uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

// Workspace pieces of one single-matrix shrinkage.
struct SvtWs {
    int64_t ldp = 0;
    float *T = nullptr;                 // sparsify transform (when requested)
    float *eps = nullptr;
    double *removed2 = nullptr;         // |Phi - Phi_|_F^2 (guarded interval)
    unsigned long long *counts = nullptr;
    float *G = nullptr, *A = nullptr, *Z[2] = {nullptr, nullptr}, *H = nullptr, *v0 = nullptr, *v1 = nullptr;
    double *out = nullptr, *norm2 = nullptr, *coef = nullptr;
    int *flag = nullptr;
    // tensor-core operands
    __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr, *Zhi[2] = {}, *Zlo[2] = {}, *Hhi = nullptr, *Hlo = nullptr;
    __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr, *Xthi = nullptr, *Xtlo = nullptr;
    int64_t ldn = 0, ldm = 0;
    // row stride of the recurrence operands (A-tilde, Psi copies): p rounded
    // up to 128, the columns beyond p kept zero so the products run over a
    // contraction length that the grouped operand loads take whole
    int64_t ldk = 0;
    // learned order: lower-edge vectors, FP64 accumulators and coefficient
    // scratch, the chosen {L, fallback}
    float *u0 = nullptr, *u1 = nullptr;
    double *lacc = nullptr, *ltab = nullptr;
    int *Lsel = nullptr;
    // tile occupancy of the thresholded operand (sparsity-based reduction)
    uint8_t *amask = nullptr;
    // compaction of the thresholded operand: row flags, the support S, {s},
    // the series' value on the zero block
    int *sflags = nullptr, *sidx = nullptr, *sinfo = nullptr;
    double *cout = nullptr;
    size_t bytes = 0;
};

SvtWs carve(char *base, int64_t m, int64_t n, int L, int iters, int prec, bool sparse = false, bool learn = false,
            bool gram_only = false) {
    SvtWs w;
    int64_t p = std::min(m, n);
    w.ldp = round_up(p, 8);
    size_t pp = (size_t)(p * w.ldp);
    Carver c(base);
    w.out = c.take<double>(8);
    w.norm2 = c.take<double>(iters + 2);
    w.coef = c.take<double>(std::max(L, 2));
    w.flag = c.take<int>(8);   // barrier and error words: 0, 1 bound; 2 recurrence; 3, 4 top-k; 5 tensor-core waits
    if (learn) {
        const size_t nacc = learn_scratch_doubles(L);
        w.lacc = c.take<double>(nacc + 2 * (size_t)L + 8);
        w.ltab = w.lacc + nacc;
        w.u0 = c.take<float>(round_up(p, 4));
        w.u1 = c.take<float>(round_up(p, 4));
        w.Lsel = c.take<int>(4);
    }
    w.G = c.take<float>(pp);
    w.A = c.take<float>(pp);
    w.Z[0] = c.take<float>(pp);
    w.Z[1] = c.take<float>(pp);
    w.H = c.take<float>(pp);
    w.v0 = c.take<float>(round_up(p, 4));
    w.v1 = c.take<float>(round_up(p, 4));
    if (gram_only && prec != CPA_FP32) {
        // the Gram step's operands only (features of a matrix)
        w.ldn = round_up(n, 8);
        w.ldm = round_up(m, 8);
        w.Xhi = c.take<__nv_bfloat16>((size_t)(m * w.ldn));
        w.Xlo = c.take<__nv_bfloat16>((size_t)(m * w.ldn));
        w.Xthi = c.take<__nv_bfloat16>((size_t)(n * w.ldm));
        w.Xtlo = c.take<__nv_bfloat16>((size_t)(n * w.ldm));
        w.bytes = c.off;
        return w;
    }
    if (sparse) {
        w.T = c.take<float>(pp);
        w.eps = c.take<float>(4);
        w.removed2 = c.take<double>(2);
        w.counts = c.take<unsigned long long>(kTopkCounts);
        w.sflags = c.take<int>(round_up(p, 4));
        w.sidx = c.take<int>(round_up(p, 4));
        w.sinfo = c.take<int>(4);
        w.cout = c.take<double>(2);
    }
    if (prec != CPA_FP32) {
        // Gram and final product always use the hi/lo split (their BF16
        // rounding would otherwise dominate the error); the recurrence
        // operands carry a lo part only in the all-split mode.
        // (the transform products of the sparsity reduction use the lo parts too)
        bool split_rec = prec == CPA_BF16X3 || p < kSplitRecBelow || sparse;
        w.ldn = round_up(n, 8);
        w.ldm = round_up(m, 8);
        w.ldk = round_up(p, 128);
        const size_t pk = (size_t)(p * w.ldk);
        w.Ahi = c.take<__nv_bfloat16>(pk);
        w.Zhi[0] = c.take<__nv_bfloat16>(pk);
        w.Zhi[1] = c.take<__nv_bfloat16>(pk);
        w.Hhi = c.take<__nv_bfloat16>(pp);
        w.Hlo = c.take<__nv_bfloat16>(pp);
        w.Xhi = c.take<__nv_bfloat16>((size_t)(m * w.ldn));
        w.Xlo = c.take<__nv_bfloat16>((size_t)(m * w.ldn));
        w.Xthi = c.take<__nv_bfloat16>((size_t)(n * w.ldm));
        w.Xtlo = c.take<__nv_bfloat16>((size_t)(n * w.ldm));
        if (split_rec) {
            w.Alo = c.take<__nv_bfloat16>(pk);
            w.Zlo[0] = c.take<__nv_bfloat16>(pk);
            w.Zlo[1] = c.take<__nv_bfloat16>(pk);
        }
        if (sparse) w.amask = c.take<uint8_t>((size_t)((p + 127) / 128) * (size_t)((w.ldk + 63) / 64));
    }
    w.bytes = c.off;
    return w;
}

cpa_status set_device(cpa_ctx *h) {
    CK(cudaSetDevice(h->device));
    return CPA_OK;
}

}  // namespace

extern "C" {

const char *cpa_status_string(cpa_status s) {
    switch (s) {
        case CPA_OK: return "ok";
        case CPA_ERR_INVALID_ARG: return "invalid argument";
        case CPA_ERR_CUDA: return "CUDA error";
        case CPA_ERR_NO_MEMORY: return "out of device memory";
        case CPA_ERR_NONFINITE: return "non-finite value in input or bound";
        case CPA_ERR_BOUND: return "invalid lambda_max bound";
        case CPA_ERR_TIMEOUT: return "device-side wait timed out";
        case CPA_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char *cpa_last_error(void) { return g_err; }

cpa_status cpa_create(cpa_handle *out, int device) {
    if (!out) return CPA_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return CPA_ERR_INVALID_ARG;
    cpa_ctx *h = new cpa_ctx();
    h->device = device;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDeviceProperties");
    }
    h->num_sms = prop.multiProcessorCount;
    h->cc = prop.major * 10 + prop.minor;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_pin, 64 * sizeof(double));
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaMallocHost");
    }
    *out = h;
    return CPA_OK;
}

cpa_status cpa_destroy(cpa_handle h) {
    if (!h) return CPA_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    for (auto &p : h->pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    if (h->stage) cudaFree(h->stage);
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    for (int i = 0; i < 2; ++i) {
        if (h->in_ready[i]) cudaEventDestroy(h->in_ready[i]);
        if (h->computed[i]) cudaEventDestroy(h->computed[i]);
        if (h->out_done[i]) cudaEventDestroy(h->out_done[i]);
    }
    if (h->start) cudaEventDestroy(h->start);
    ptr_plan_destroy(h->pplan);
    ptr_plan_destroy(h->pplan_tc);
    for (int k = 0; k < kMaxStreams; ++k) {
        if (h->sub[k]) cpa_destroy(h->sub[k]);
        if (h->sub_st[k]) cudaStreamDestroy(h->sub_st[k]);
        if (h->sub_ev[k]) cudaEventDestroy(h->sub_ev[k]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->d_big_L) cudaFree(h->d_big_L);
    if (h->d_big_lam) cudaFree(h->d_big_lam);
    delete h;
    return CPA_OK;
}

cpa_status cpa_coeffs(const cpa_shrink *s, int L, double lambda_max, double *c_out) {
    if (check_shrink(s) != CPA_OK || L < 1 || L > kMaxTerms || !(lambda_max > 0.0) ||
        !std::isfinite(lambda_max) || !c_out)
        return CPA_ERR_INVALID_ARG;
    ShrinkParams p = to_params(s);
    for (int k = 0; k < L; ++k) {
        double acc = 0.0;
        for (int l = 1; l <= L; ++l) {
            double th = kPi * ((double)l - 0.5) / (double)L;
            double x = 0.5 * lambda_max * (cos(th) + 1.0);
            acc += cos((double)k * th) * response(p, x);
        }
        c_out[k] = 2.0 / (double)L * acc;
    }
    return CPA_OK;
}

}  // extern "C"

namespace {

// Gram matrix of the smaller side into w.G (FP32 accumulate).
cpa_status run_gram(cpa_ctx *h, const float *dX, int64_t m, int64_t n, int64_t ldx, const SvtWs &w, int prec,
                    cudaStream_t st) {
    int64_t p = std::min(m, n);
    Epilogue e;
    e.D = w.G;
    e.ldd = w.ldp;
    if (prec == CPA_FP32) {
        e.symmetric_upper = 1;
        if (m >= n)   // G = X^T X: A(i,k) = X[k][i]
            CK(gemm_f32((int)p, (int)p, (int)m, dX, ldx, false, dX, ldx, false, e, st));
        else          // G = X X^T
            CK(gemm_f32((int)p, (int)p, (int)n, dX, ldx, true, dX, ldx, true, e, st));
        return CPA_OK;
    }
    // tensor cores: K-major BF16 hi/lo operand of the contraction dimension;
    // upper tiles only, mirrored, so G is exactly symmetric
    const int nsplit = 3;
    e.symmetric_upper = 1;
    e.sym_full_d = 1;   // G is read in full by the power iteration and the shift
    e.err = w.flag + 5;
    TcOperand op;
    if (m >= n) {   // rows of X^T (n x m)
        op.hi = w.Xthi; op.lo = w.Xtlo; op.ld = w.ldm; op.rows = (int)n;
        CK(gemm_tc((int)p, (int)p, (int)m, op, op, nsplit, e, st, h->num_sms));
    } else {
        op.hi = w.Xhi; op.lo = w.Xlo; op.ld = w.ldn; op.rows = (int)m;
        CK(gemm_tc((int)p, (int)p, (int)n, op, op, nsplit, e, st, h->num_sms));
    }
    return CPA_OK;
}

cpa_status validate_matrix(const float *dX, int64_t m, int64_t n, int64_t ldx) {
    if (!dX || m < 1 || n < 1 || ldx < n) return CPA_ERR_INVALID_ARG;
    if (std::min(m, n) > 32768 || std::max(m, n) > (int64_t)1 << 24) return CPA_ERR_INVALID_ARG;
    return CPA_OK;
}

}  // namespace

extern "C" {

cpa_status cpa_lambda_bound(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx, int iters,
                            double *lambda_out, void *stream) {
    if (!h || !lambda_out || iters < 0 || iters > 100000) return CPA_ERR_INVALID_ARG;
    cpa_status s = validate_matrix(dX, m, n, ldx);
    if (s != CPA_OK) return s;
    if ((s = set_device(h)) != CPA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    SvtWs w = carve(nullptr, m, n, 1, iters, CPA_FP32);
    if ((s = ensure_ws(h, w.bytes, st)) != CPA_OK) return s;
    w = carve(h->ws, m, n, 1, iters, CPA_FP32);
    int64_t p = std::min(m, n);
    if ((s = run_gram(h, dX, m, n, ldx, w, CPA_FP32, st)) != CPA_OK) return s;
    CK(power_bound_persistent(w.G, w.ldp, (int)p, iters, w.v0, w.v1, w.norm2, (unsigned int *)w.flag, w.flag + 1,
                              w.out, st, h->num_sms, 0, nullptr, nullptr, h->wait));
    CK(cudaMemcpyAsync(h->h_pin, w.out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->h_pin[4] != 0.0) return (cpa_status)(int)h->h_pin[4];
    *lambda_out = h->h_pin[3];
    return CPA_OK;
}

}  // extern "C"

namespace {

// The learned choice of (Lambda_max, L): the network's parameters and the
// decision rule.
struct LearnCall {
    const float *P;
    cpa_learn_rule rule;
};

cpa_status svt_impl(cpa_ctx *h, const float *dX, int64_t m, int64_t n, int64_t ldx, const cpa_shrink *sh, int L,
                    double lambda_max, int prec, const cpa_sparsify *sp, float *dY, int64_t ldy, void *stream,
                    const LearnCall *learn);

}  // namespace

extern "C" {

cpa_status cpa_svt(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx, const cpa_shrink *sh,
                   int L, double lambda_max, int prec, const cpa_sparsify *sp, float *dY, int64_t ldy,
                   void *stream) {
    return svt_impl(h, dX, m, n, ldx, sh, L, lambda_max, prec, sp, dY, ldy, stream, nullptr);
}

cpa_status cpa_svt_learned(cpa_handle h, cpa_mlp net, const float *dX, int64_t m, int64_t n, int64_t ldx,
                           const cpa_shrink *sh, const cpa_learn_rule *rule, int prec, float *dY, int64_t ldy,
                           void *stream) {
    if (!h || !net || !rule) return CPA_ERR_INVALID_ARG;
    const cpa_learn_rule &r = *rule;
    if (!(r.L_scale > 0.0) || !std::isfinite(r.L_scale) || !(r.margin >= 0.0) || !std::isfinite(r.margin) ||
        r.L_min < 1 || r.L_max < r.L_min || r.L_max > kMaxTerms || r.L_fallback < 1 || r.L_fallback > r.L_max)
        return CPA_ERR_INVALID_ARG;
    int dims[4], dev = -1;
    const float *P = mlp_device_params(net, dims, &dev);
    if (!P || dims[0] != 12 || dims[1] != 64 || dims[2] != 64 || dims[3] != 2 || dev != h->device)
        return CPA_ERR_INVALID_ARG;   // the 12 -> 64 -> 64 -> 2 predictor, on the handle's device
    if (h->series != CPA_SERIES_FORWARD) return CPA_ERR_UNSUPPORTED;
    LearnCall lc{P, r};
    return svt_impl(h, dX, m, n, ldx, sh, r.L_max, 0.0, prec, nullptr, dY, ldy, stream, &lc);
}

cpa_status cpa_get_order(cpa_handle h, int *L_out, int *fallback, void *stream) {
    if (!h || !h->have_learn || (!L_out && !fallback)) return CPA_ERR_INVALID_ARG;
    cpa_status s = set_device(h);
    if (s != CPA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int *pin = reinterpret_cast<int *>(h->h_pin + 8);
    CK(cudaMemcpyAsync(pin, h->d_L, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (L_out) *L_out = pin[0];
    if (fallback) *fallback = pin[1];
    return CPA_OK;
}

cpa_status cpa_learn_features(cpa_handle h, const float *dX, int64_t m, int64_t n, int64_t ldx,
                              const cpa_shrink *sh, float *dF, double *dTheta, void *stream) {
    if (!h || !dF || !dTheta) return CPA_ERR_INVALID_ARG;
    cpa_status s = validate_matrix(dX, m, n, ldx);
    if (s != CPA_OK) return s;
    if ((s = check_shrink(sh)) != CPA_OK) return s;
    if ((s = set_device(h)) != CPA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = h->cc >= 100 ? CPA_BF16X3 : CPA_FP32;
    SvtWs w = carve(nullptr, m, n, 2, 4, prec, false, true, true);
    if ((s = ensure_ws(h, w.bytes, st)) != CPA_OK) return s;
    w = carve(h->ws, m, n, 2, 4, prec, false, true, true);
    const int64_t p = std::min(m, n);
    if (prec != CPA_FP32) {
        CK(split_bf16(dX, (int)m, (int)n, ldx, false, w.Xhi, w.Xlo, w.ldn, st));
        CK(split_bf16(dX, (int)m, (int)n, ldx, true, w.Xthi, w.Xtlo, w.ldm, st));
    }
    CK(cudaMemsetAsync(w.flag + 5, 0, sizeof(int), st));
    if ((s = run_gram(h, dX, m, n, ldx, w, prec, st)) != CPA_OK) return s;
    ShrinkParams sp_ = to_params(sh);
    CK(learn_bound(w.G, w.ldp, (int)p, (int)std::max(m, n), sp_, nullptr, 1.0, 0.0, 1, 2, 1, 0, 1,
                   kDefaultPowerIters, w.v0, w.v1, w.u0, w.u1, w.lacc, w.ltab, (unsigned int *)w.flag, w.flag + 1,
                   w.out, w.Lsel, dF, dTheta, w.coef, st, h->num_sms, h->wait));
    return CPA_OK;
}

}  // extern "C"

namespace {

cpa_status svt_impl(cpa_ctx *h, const float *dX, int64_t m, int64_t n, int64_t ldx, const cpa_shrink *sh, int L,
                    double lambda_max, int prec, const cpa_sparsify *sp, float *dY, int64_t ldy, void *stream,
                    const LearnCall *learn) {
    if (!h || !dY || ldy < n || L < 1 || L > kMaxTerms) return CPA_ERR_INVALID_ARG;
    cpa_status s = validate_matrix(dX, m, n, ldx);
    if (s != CPA_OK) return s;
    if ((s = check_shrink(sh)) != CPA_OK) return s;
    if (!std::isfinite(lambda_max)) return CPA_ERR_INVALID_ARG;
    if (prec < CPA_FP32 || prec > CPA_BF16X3) return CPA_ERR_INVALID_ARG;
    const bool sparse = sp && (sp->transform != CPA_T_IDENTITY || sp->mode != CPA_SPARSE_OFF);
    if (sp) {
        if (sp->transform < CPA_T_IDENTITY || sp->transform > CPA_T_DCT || sp->mode < CPA_SPARSE_OFF ||
            sp->mode > CPA_SPARSE_TOPK || !std::isfinite(sp->eps_or_frac))
            return CPA_ERR_INVALID_ARG;
        if (sp->mode == CPA_SPARSE_ABS && !(sp->eps_or_frac >= 0.0)) return CPA_ERR_INVALID_ARG;
        if (sp->mode == CPA_SPARSE_TOPK && !(sp->eps_or_frac > 0.0 && sp->eps_or_frac <= 1.0))
            return CPA_ERR_INVALID_ARG;
        if (sp->interval != 0 && sp->interval != 1) return CPA_ERR_INVALID_ARG;
    }
    const bool guarded = sparse && sp->interval == 1 && sp->mode != CPA_SPARSE_OFF;
    if (ranges_overlap(dX, (size_t)((m - 1) * ldx + n) * sizeof(float), dY,
                       (size_t)((m - 1) * ldy + n) * sizeof(float)))
        return CPA_ERR_INVALID_ARG;
    if (prec != CPA_FP32 && h->cc < 100) return CPA_ERR_UNSUPPORTED;
    if (prec == CPA_TF32) return CPA_ERR_UNSUPPORTED;
    // Clenshaw's intermediates are larger than the filter they sum to, so a
    // plain BF16 operand per step costs about fifty times the forward
    // recurrence's error, above the BF16 path's 2e-3 bar: not offered
    if (h->series == CPA_SERIES_CLENSHAW && prec == CPA_BF16) return CPA_ERR_UNSUPPORTED;
    if ((s = set_device(h)) != CPA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int iters = kDefaultPowerIters;
    SvtWs w = carve(nullptr, m, n, L, iters, prec, sparse, learn != nullptr);
    if ((s = ensure_ws(h, w.bytes, st)) != CPA_OK) return s;
    w = carve(h->ws, m, n, L, iters, prec, sparse, learn != nullptr);
    // the call's error word (timeouts of the tensor-core kernels' waits),
    // read back by cpa_get_lambda and cpa_sync_status
    h->d_err = w.flag + 5;
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    const int64_t p = std::min(m, n);
    const bool tc = prec != CPA_FP32;
    // Gram and final product: always split.  Recurrence: split in BF16X3
    // mode, and for small p in BF16 mode too (there the products are
    // latency-bound, and a single BF16 rounding of a tiny matrix is not
    // averaged out).
    const int nsplit_rec = (prec == CPA_BF16X3 || p < kSplitRecBelow) ? 3 : 1;
    const int clenshaw = h->series == CPA_SERIES_CLENSHAW ? 1 : 0;
    ShrinkParams sp_ = to_params(sh);

    // operand preparation for the tensor-core path: X and X^T as BF16 hi/lo
    if (tc) {
        StageScope sc(h, CPA_STAGE_PREP, st, 2);
        CK(split_bf16(dX, (int)m, (int)n, ldx, false, w.Xhi, w.Xlo, w.ldn, st));
        CK(split_bf16(dX, (int)m, (int)n, ldx, true, w.Xthi, w.Xtlo, w.ldm, st));
    }
    // Gram step
    {
        StageScope sc(h, CPA_STAGE_GRAM, st, 1);
        if ((s = run_gram(h, dX, m, n, ldx, w, prec, st)) != CPA_OK) return s;
    }
    // sparsity-based reduction: Phi = T G T^T, entries below eps set to zero
    if (sparse) {
        StageScope sc(h, CPA_STAGE_SPARSE, st, 0);
        CK(make_transform(sp->transform, (int)p, w.T, w.ldp, st, h->num_sms, w.Z[1]));   // Z[1]: free scratch
        Epilogue e1;
        e1.D = w.A;   // T G (w.A is free until the shift)
        e1.ldd = w.ldp;
        Epilogue e2;
        e2.D = w.G;   // (T G) T^T, exactly symmetric
        e2.ldd = w.ldp;
        e2.symmetric_upper = 1;
        if (!tc) {
            CK(gemm_f32((int)p, (int)p, (int)p, w.T, w.ldp, true, w.G, w.ldp, true, e1, st));
            CK(gemm_f32((int)p, (int)p, (int)p, w.A, w.ldp, true, w.T, w.ldp, true, e2, st));
            h->launches[CPA_STAGE_SPARSE] += 3;
        } else {
            // on the tensor cores with the hi/lo split: rows of T and of G
            // (symmetric) give T G; rows of T G and of T give (T G) T^T
            e1.err = e2.err = w.flag + 5;
            e2.sym_full_d = 1;
            CK(split_bf16(w.T, (int)p, (int)p, w.ldp, false, w.Zhi[0], w.Zlo[0], w.ldk, st));
            CK(split_bf16(w.G, (int)p, (int)p, w.ldp, false, w.Zhi[1], w.Zlo[1], w.ldk, st));
            TcOperand tr, gr, tg;
            tr.hi = w.Zhi[0]; tr.lo = w.Zlo[0]; tr.ld = w.ldk; tr.rows = (int)p;
            gr.hi = w.Zhi[1]; gr.lo = w.Zlo[1]; gr.ld = w.ldk; gr.rows = (int)p;
            CK(gemm_tc((int)p, (int)p, (int)p, tr, gr, 3, e1, st, h->num_sms));
            CK(split_bf16(w.A, (int)p, (int)p, w.ldp, false, w.Ahi, w.Alo, w.ldk, st));
            tg.hi = w.Ahi; tg.lo = w.Alo; tg.ld = w.ldk; tg.rows = (int)p;
            CK(gemm_tc((int)p, (int)p, (int)p, tg, tr, 3, e2, st, h->num_sms));
            h->launches[CPA_STAGE_SPARSE] += 6;
        }
        if (guarded) CK(cudaMemsetAsync(w.removed2, 0, sizeof(double), st));
        // the threshold also marks the rows that keep a nonzero entry (the
        // compaction's support)
        int *rf = (sp->mode != CPA_SPARSE_OFF && !learn && h->sparse_compact && iters >= 1) ? w.sflags : nullptr;
        if (sp->mode == CPA_SPARSE_ABS) {
            CK(threshold_entries(w.G, (int)p, w.ldp, nullptr, (float)sp->eps_or_frac, st, h->num_sms,
                                 guarded ? w.removed2 : nullptr, rf));
            h->launches[CPA_STAGE_SPARSE] += 1;
        } else if (sp->mode == CPA_SPARSE_TOPK) {
            const double pp2 = (double)p * (double)p;
            long long k = (long long)std::ceil(sp->eps_or_frac * pp2);
            k = std::max(1LL, std::min(k, (long long)pp2));
            CK(topk_eps(w.G, (int)p, w.ldp, k, w.counts, (unsigned int *)(w.flag + 3), w.flag + 4, w.eps, st,
                        h->num_sms));
            CK(threshold_entries(w.G, (int)p, w.ldp, w.eps, 0.f, st, h->num_sms, guarded ? w.removed2 : nullptr,
                                 rf));
            h->launches[CPA_STAGE_SPARSE] += 2;
        }
    }
    // compaction: when the thresholded operand's nonzero rows S are at most
    // half of them, the bound, shift and recurrence run on the |S| x |S|
    // block Phi_[S, S] (its polynomials are those of Phi_ on S and a
    // constant elsewhere; sparsify.cu's header); one synchronisation reads |S|
    int64_t pr = p;   // the order of the matrix the series is built on
    bool compact = false;
    if (sparse && sp->mode != CPA_SPARSE_OFF && !learn && h->sparse_compact && iters >= 1) {
        StageScope sc(h, CPA_STAGE_SPARSE, st, 1);
        CK(compact_support(w.sflags, (int)p, w.sidx, w.sinfo, st));
        int *pin = reinterpret_cast<int *>(h->h_pin + 10);
        CK(cudaMemcpyAsync(pin, w.sinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int sdim = pin[0];
        if (sdim >= 1 && 2 * (int64_t)sdim <= p) {
            compact = true;
            pr = sdim;
            CK(gather_block(w.G, w.ldp, w.sidx, sdim, w.Z[0], w.ldp, st, h->num_sms));
            CK(cudaMemcpy2DAsync(w.G, (size_t)w.ldp * sizeof(float), w.Z[0], (size_t)w.ldp * sizeof(float),
                                 (size_t)sdim * sizeof(float), (size_t)sdim, cudaMemcpyDeviceToDevice, st));
            h->launches[CPA_STAGE_SPARSE] += 1;
        }
    }
    // interval bound
    if (learn) {
        // features, network, decision and the chosen order's coefficients in
        // one launch; L stays on the device for the recurrence
        StageScope sc(h, CPA_STAGE_BOUND, st, 1);
        const cpa_learn_rule &r = learn->rule;
        CK(learn_bound(w.G, w.ldp, (int)p, (int)std::max(m, n), sp_, learn->P, r.L_scale, r.margin, r.L_min, r.L_max,
                       r.L_fallback, r.use_lambda, 0, iters, w.v0, w.v1, w.u0, w.u1, w.lacc, w.ltab,
                       (unsigned int *)w.flag, w.flag + 1, w.out, w.Lsel, nullptr, nullptr, w.coef, st, h->num_sms,
                       h->wait));
    } else if (lambda_max > 0.0) {
        StageScope sc(h, CPA_STAGE_BOUND, st, 1);
        set_scalar2_kernel<<<1, 1, 0, st>>>(w.out + 3, lambda_max, 0.0);
        CK(cudaGetLastError());
    } else {
        // the bound's launch also forms the coefficients (FP64) in its last block
        StageScope sc(h, CPA_STAGE_BOUND, st, 1);
        CK(power_bound_persistent(w.G, w.ldp, (int)pr, iters, w.v0, w.v1, w.norm2, (unsigned int *)w.flag,
                                  w.flag + 1, w.out, st, h->num_sms, L, &sp_, w.coef, h->wait,
                                  compact ? w.sidx : nullptr));
    }
    // guarded interval [-|Phi - Phi_|_F, Lambda_max]: its ends are read
    // once (one synchronisation) and its coefficients formed on the host
    double span = 0.0, sigma = 1.0;
    if (guarded) {
        CK(cudaMemcpyAsync(h->h_pin, w.out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h->h_pin + 6, w.removed2, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double b = h->h_pin[3], a = -sqrt(std::max(h->h_pin[6], 0.0));
        if (!(b > 0.0) || !std::isfinite(b) || !std::isfinite(a)) return CPA_ERR_BOUND;
        span = b - a;
        sigma = (a + b) / (b - a);
        std::vector<double> cc((size_t)L);
        coeffs_interval(sp_, L, a, b, cc.data());
        CK(cudaMemcpy(w.coef, cc.data(), sizeof(double) * (size_t)L, cudaMemcpyHostToDevice));
    }
    // coefficients (FP64, on the device so the call stays asynchronous)
    if (lambda_max > 0.0 && !learn && !guarded) {
        StageScope sc(h, CPA_STAGE_COEFF, st, 1);
        CK(device_coeffs(w.out + 3, 0.0, L, sp_, w.coef, st));
    }
    // shift and initial sum; Psi_1 = B_hat lives in ring slot 1
    {
        StageScope sc(h, CPA_STAGE_SHIFT, st, 1);
        CK(shift_init(w.G, w.ldp, (int)pr, w.out + 3, w.coef, L, tc ? nullptr : w.A, w.Z[1], w.H, w.ldp,
                      tc ? w.Ahi : nullptr, tc ? w.Alo : nullptr, tc ? w.Zhi[1] : nullptr,
                      tc ? w.Zlo[1] : nullptr, tc ? w.ldk : w.ldp, st, h->num_sms, clenshaw,
                      tc ? w.Zhi[0] : nullptr, tc ? w.Zlo[0] : nullptr, span, sigma));
    }
    // recurrence with fused accumulation: Psi_k = 2 B_hat Psi_{k-1} - Psi_{k-2}, H += c_k Psi_k.
    // Ring: Psi_k overwrites Psi_{k-2} in slot k&1; Psi_0 = Id is implicit.
    // Both paths multiply by At = (2/lambda) G and apply the shift exactly
    // in the FP32 epilogue:  Psi_k = 2 At Psi_{k-1} - 2 Psi_{k-1} - Psi_{k-2}.
    int closed = 0;   // Clenshaw's closing step already applied by the launch
    if (tc && L > 2) {
        // every step in one cooperative launch (grid barrier between steps)
        StageScope sc(h, CPA_STAGE_RECUR, st, 1);
        Epilogue e;
        e.D = w.Z[0];
        e.ldd = w.ldp;
        e.ldc = w.ldp;
        e.ldc2 = w.ldp;
        e.s_acc = 2.f;
        e.s_c = -1.f;
        e.s_c2 = (float)(-2.0 * sigma);
        e.H = w.H;
        e.ldh = w.ldp;
        e.coef = w.coef;
        e.ldb = w.ldk;
        e.symmetric_upper = 1;
        e.err = w.flag + 5;
        TcOperand a;
        a.hi = w.Ahi; a.lo = w.Alo; a.ld = w.ldk; a.rows = (int)pr;
        CK(gemm_tc_recurrence((int)pr, a, nsplit_rec, e, 2, L, w.Z, w.Zhi, w.Zlo, (unsigned int *)(w.flag + 2), st,
                              h->num_sms, clenshaw, L, &closed, compact ? (int)round_up(pr, 128) : (int)w.ldk,
                              h->wait, learn ? w.Lsel : nullptr,
                              (sparse && sp->mode != CPA_SPARSE_OFF && h->sparse_skip && !compact) ? w.amask
                                                                                                    : nullptr));
    }
    if (learn && !tc) {
        // the CUDA-core recurrence is driven from the host: read the order
        int *pin = reinterpret_cast<int *>(h->h_pin + 8);
        CK(cudaMemcpyAsync(pin, w.Lsel, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        L = std::max(1, std::min(L, pin[0]));
    }
    for (int k = 2; k < L && !tc; ++k) {
        StageScope sc(h, CPA_STAGE_RECUR, st, 1);
        Epilogue e;
        int cur = k & 1, prev = (k - 1) & 1;
        e.D = w.Z[cur];
        e.ldd = w.ldp;
        e.C = (k == 2) ? nullptr : w.Z[cur];   // Psi_{k-2}
        e.ldc = w.ldp;
        e.s_acc = 2.f;
        e.s_c = -1.f;
        e.diag = (k == 2) ? -1.f : 0.f;        // - Psi_0 = - Id
        e.H = w.H;
        e.ldh = w.ldp;
        e.coef = w.coef;
        e.k = k;
        e.symmetric_upper = 1;
        if (clenshaw) {
            // b_kk = 2 B_hat b_{kk+1} - b_{kk+2} + c_kk Id, kk = L-1-k; b_{L-1} =
            // c_{L-1} Id enters the first step on the diagonal; b_0 goes to H
            const int kk = L - 1 - k;
            e.D = kk == 0 ? w.H : w.Z[cur];
            e.diag = 0.f;
            e.dcoef = w.coef;
            e.dk = kk;
            e.dk2 = (k == 2) ? L - 1 : -1;
            e.H = nullptr;
        }
        if (!tc) {
            // A holds At = (2/lambda) G: the -Id of B_hat is applied here
            // exactly, -2 Psi_{k-1} (FP32 rounding of B_hat's diagonal near
            // -1 would move the eigenvalues near the interval's ends)
            e.C2 = w.Z[prev];
            e.ldc2 = w.ldp;
            e.s_c2 = (float)(-2.0 * sigma);
            CK(gemm_f32((int)pr, (int)pr, (int)pr, w.A, w.ldp, true, w.Z[prev], w.ldp, true, e, st));
        } else {
            e.C2 = w.Z[prev];                  // Psi_{k-1}
            e.ldc2 = w.ldp;
            e.s_c2 = (float)(-2.0 * sigma);
            e.Dhi = w.Zhi[cur];
            e.Dlo = w.Zlo[cur];
            e.ldb = w.ldk;
            e.err = w.flag + 5;
            TcOperand a, b;
            a.hi = w.Ahi; a.lo = w.Alo; a.ld = w.ldk; a.rows = (int)pr;
            b.hi = w.Zhi[prev]; b.lo = w.Zlo[prev]; b.ld = w.ldk; b.rows = (int)pr;
            CK(gemm_tc((int)pr, (int)pr, (int)pr, a, b, nsplit_rec, e, st, h->num_sms));
        }
    }
    // Clenshaw's closing step: H = (b_0 - b_2) / 2, b_2 in ring slot (L-1)&1
    // (L = 3: b_2 = c_2 Id); the tensor-core path keeps the lower triangle
    if (clenshaw && L >= 3 && !closed) {
        StageScope sc(h, CPA_STAGE_RECUR, st, 1);
        CK(clenshaw_finish(w.H, L == 3 ? nullptr : w.Z[(L - 1) & 1], (int)pr, w.ldp, w.coef, tc ? 1 : 0, st,
                           h->num_sms));
    }
    // with the sparsity option the filter applied to X is T^T H T (Eq. SVD_fil)
    float *Hf = w.H;
    if (sparse && compact) {
        // T^T H T = T_S^T (H_hat(A) - c_out Id) T_S + c_out T^T T
        StageScope sc(h, CPA_STAGE_SPARSE, st, 6 + (tc ? 1 : 0));
        if (tc) CK(symmetrize_lower(w.H, (int)pr, w.ldp, st, h->num_sms));
        const double sig = guarded ? sigma : 1.0;
        CK(zero_block_value(w.coef, L, sig, w.cout, st));
        CK(diag_add(w.H, (int)pr, w.ldp, w.cout, -1.0, st));
        CK(gather_rows(w.T, w.ldp, w.sidx, (int)pr, (int)p, w.Z[0], w.ldp, st, h->num_sms));
        Epilogue ew;
        ew.D = w.Z[1];   // (H_hat(A) - c_out Id) T_S, |S| x p
        ew.ldd = w.ldp;
        CK(gemm_f32((int)pr, (int)p, (int)pr, w.H, w.ldp, true, w.Z[0], w.ldp, false, ew, st));
        Epilogue ef;
        ef.D = w.A;      // T_S^T (...) T_S, p x p, exactly symmetric
        ef.ldd = w.ldp;
        ef.symmetric_upper = 1;
        CK(gemm_f32((int)p, (int)p, (int)pr, w.Z[0], w.ldp, false, w.Z[1], w.ldp, false, ef, st));
        CK(add_transform_gram(w.A, (int)p, w.ldp, sp->transform, w.cout, st));
        Hf = w.A;
    } else if (sparse) {
        StageScope sc(h, CPA_STAGE_SPARSE, st, tc ? 6 : 2);
        Epilogue e1;
        e1.D = w.Z[0];   // T^T H
        e1.ldd = w.ldp;
        Epilogue e2;
        e2.D = w.Z[1];   // (T^T H) T
        e2.ldd = w.ldp;
        e2.symmetric_upper = 1;
        if (!tc) {
            CK(gemm_f32((int)p, (int)p, (int)p, w.T, w.ldp, false, w.H, w.ldp, true, e1, st));
            CK(gemm_f32((int)p, (int)p, (int)p, w.Z[0], w.ldp, true, w.T, w.ldp, false, e2, st));
        } else {
            // tensor cores: rows of T^T and of H (symmetric) give T^T H; rows
            // of T^T H and of T^T give (T^T H) T
            CK(symmetrize_lower(w.H, (int)p, w.ldp, st, h->num_sms));
            e1.err = e2.err = w.flag + 5;
            e2.sym_full_d = 1;
            CK(split_bf16(w.T, (int)p, (int)p, w.ldp, true, w.Zhi[0], w.Zlo[0], w.ldk, st));
            CK(split_bf16(w.H, (int)p, (int)p, w.ldp, false, w.Zhi[1], w.Zlo[1], w.ldk, st));
            TcOperand ttr, hr, th;
            ttr.hi = w.Zhi[0]; ttr.lo = w.Zlo[0]; ttr.ld = w.ldk; ttr.rows = (int)p;
            hr.hi = w.Zhi[1]; hr.lo = w.Zlo[1]; hr.ld = w.ldk; hr.rows = (int)p;
            CK(gemm_tc((int)p, (int)p, (int)p, ttr, hr, 3, e1, st, h->num_sms));
            CK(split_bf16(w.Z[0], (int)p, (int)p, w.ldp, false, w.Ahi, w.Alo, w.ldk, st));
            th.hi = w.Ahi; th.lo = w.Alo; th.ld = w.ldk; th.rows = (int)p;
            CK(gemm_tc((int)p, (int)p, (int)p, th, ttr, 3, e2, st, h->num_sms));
        }
        Hf = w.Z[1];
    }
    // final product: Y = X H (m >= n) or H X (m < n)
    StageScope sc(h, CPA_STAGE_APPLY, st, tc ? 2 : 1);
    Epilogue e;
    e.D = dY;
    e.ldd = ldy;
    e.err = w.flag + 5;
    if (!tc) {
        if (m >= n)
            CK(gemm_f32((int)m, (int)n, (int)n, dX, ldx, true, Hf, w.ldp, true, e, st));
        else
            CK(gemm_f32((int)m, (int)n, (int)m, Hf, w.ldp, true, dX, ldx, false, e, st));
    } else {
        // H is valid in its lower triangle (the tensor-core epilogue keeps
        // the FP32 arrays there); the split writes both triangles.  The
        // transformed filter is full and split as it is.
        if (sparse)
            CK(split_bf16(Hf, (int)p, (int)p, w.ldp, false, w.Hhi, w.Hlo, w.ldp, st));
        else
            CK(split_sym_lower(w.H, (int)p, w.ldp, w.Hhi, w.Hlo, w.ldp, st));
        TcOperand hop, xop;
        hop.hi = w.Hhi; hop.lo = w.Hlo; hop.ld = w.ldp; hop.rows = (int)p;
        if (m >= n) {   // Y(r,j) = sum_l X[r][l] H[j][l]
            xop.hi = w.Xhi; xop.lo = w.Xlo; xop.ld = w.ldn; xop.rows = (int)m;
            CK(gemm_tc((int)m, (int)n, (int)n, xop, hop, 3, e, st, h->num_sms));
        } else {        // Y(i,c) = sum_l H[i][l] X^T[c][l]
            xop.hi = w.Xthi; xop.lo = w.Xtlo; xop.ld = w.ldm; xop.rows = (int)n;
            CK(gemm_tc((int)m, (int)n, (int)m, hop, xop, 3, e, st, h->num_sms));
        }
    }
    h->d_out = w.out;
    h->d_coef = w.coef;
    h->last_L = learn ? learn->rule.L_max : L;
    h->have_last = true;
    h->have_learn = learn != nullptr;
    h->d_L = learn ? w.Lsel : nullptr;
    return CPA_OK;
}

}  // namespace

extern "C" {

// Reads {theta, r, trace, lambda, status} of the last cpa_svt and its
// tensor-core error word into the handle's pinned slots (synchronises).
static cpa_status read_last(cpa_ctx *h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->h_pin, h->d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_pin + 5, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return CPA_OK;
}

static cpa_status last_status(const cpa_ctx *h) {
    int err = 0;
    memcpy(&err, h->h_pin + 5, sizeof(int));
    if (err != 0) return (cpa_status)err;
    if (h->h_pin[4] != 0.0) return (cpa_status)(int)h->h_pin[4];
    if (!(h->h_pin[3] > 0.0)) return CPA_ERR_BOUND;
    return CPA_OK;
}

cpa_status cpa_get_lambda(cpa_handle h, double *lambda_out, void *stream) {
    if (!h || !lambda_out || !h->have_last) return CPA_ERR_INVALID_ARG;
    cpa_status s = set_device(h);
    if (s != CPA_OK) return s;
    if ((s = read_last(h, (cudaStream_t)stream)) != CPA_OK) return s;
    *lambda_out = h->h_pin[3];
    return last_status(h);
}

cpa_status cpa_sync_status(cpa_handle h, void *stream) {
    if (!h || !h->have_last) return CPA_ERR_INVALID_ARG;
    cpa_status s = set_device(h);
    if (s != CPA_OK) return s;
    if ((s = read_last(h, (cudaStream_t)stream)) != CPA_OK) return s;
    return last_status(h);
}

cpa_status cpa_get_coeffs(cpa_handle h, double *c_out, int L, void *stream) {
    if (!h || !c_out || !h->have_last || L != h->last_L) return CPA_ERR_INVALID_ARG;
    cpa_status s = set_device(h);
    if (s != CPA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(c_out, h->d_coef, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return CPA_OK;
}

}  // extern "C"

extern "C" {

cpa_status cpa_set_option(cpa_handle h, int option, int value) {
    if (!h) return CPA_ERR_INVALID_ARG;
    if (option == CPA_OPT_SERIES) {
        if (value != CPA_SERIES_FORWARD && value != CPA_SERIES_CLENSHAW) return CPA_ERR_INVALID_ARG;
        h->series = value;
        return CPA_OK;
    }
    if (option == CPA_OPT_WAIT_KCYCLES) {
        if (value < 0) return CPA_ERR_INVALID_ARG;
        h->wait.wait_cycles = (long long)value * 1000LL;
        return CPA_OK;
    }
    if (option == CPA_OPT_STREAMS) {
        if (value < 1 || value > kMaxStreams) return CPA_ERR_INVALID_ARG;
        h->nstreams = value;
        return CPA_OK;
    }
    if (option == CPA_OPT_MEMBER_SMS) {
        if (value < 0) return CPA_ERR_INVALID_ARG;
        h->member_sms = value;
        return CPA_OK;
    }
    if (option == CPA_OPT_SPARSE_SKIP) {
        if (value != 0 && value != 1) return CPA_ERR_INVALID_ARG;
        h->sparse_skip = value;
        return CPA_OK;
    }
    if (option == CPA_OPT_SPARSE_COMPACT) {
        if (value != 0 && value != 1) return CPA_ERR_INVALID_ARG;
        h->sparse_compact = value;
        return CPA_OK;
    }
    if (option == CPA_OPT_STALL_TEST) {
        if (value != 0 && value != 1) return CPA_ERR_INVALID_ARG;
        h->wait.stall = value;
        return CPA_OK;
    }
    return CPA_ERR_INVALID_ARG;
}

cpa_status cpa_profile_enable(cpa_handle h, int enable) {
    if (!h) return CPA_ERR_INVALID_ARG;
    h->profiling = enable != 0;
    for (int k = 0; k < kMaxStreams; ++k)
        if (h->sub[k]) h->sub[k]->profiling = h->profiling;
    return CPA_OK;
}

}  // extern "C"

namespace {

// The stage times of a handle's finished event pairs into its totals.
void collect_profile(cpa_ctx *h) {
    for (auto &p : h->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) h->ms[p.first] += t;
        h->event_pool.push_back(p.second.first);
        h->event_pool.push_back(p.second.second);
    }
    h->pending.clear();
}

}  // namespace

extern "C" {

cpa_status cpa_profile_read(cpa_handle h, double *ms, int64_t *launches, int reset) {
    if (!h) return CPA_ERR_INVALID_ARG;
    cpa_status s = set_device(h);
    if (s != CPA_OK) return s;
    CK(cudaDeviceSynchronize());
    // the handle's own stages and those of its member sub-handles (members
    // of pointer-form batches run there)
    collect_profile(h);
    for (int i = 0; i < CPA_NSTAGES; ++i) {
        double t = h->ms[i];
        int64_t n = h->launches[i];
        for (int k = 0; k < kMaxStreams; ++k) {
            cpa_ctx *c = h->sub[k];
            if (!c) continue;
            if (i == 0) collect_profile(c);
            t += c->ms[i];
            n += c->launches[i];
        }
        if (ms) ms[i] = t;
        if (launches) launches[i] = n;
    }
    if (reset)
        for (int i = 0; i < CPA_NSTAGES; ++i) {
            h->ms[i] = 0.0;
            h->launches[i] = 0;
            for (int k = 0; k < kMaxStreams; ++k)
                if (h->sub[k]) {
                    h->sub[k]->ms[i] = 0.0;
                    h->sub[k]->launches[i] = 0;
                }
        }
    return CPA_OK;
}

}  // extern "C"

extern "C" {

cpa_status cpa_kernel_gemm_bf16(int M, int N, int K, const void *A_hi, const void *A_lo, int64_t lda,
                                const void *B_hi, const void *B_lo, int64_t ldb, int nsplit, int sym, float s_acc,
                                const float *C, float s_c, const float *C2, float s_c2, float diag, float *H,
                                const double *coef, int k, float *D, int64_t ldd, void *Dhi, void *Dlo, int64_t ldh,
                                void *stream) {
    if (M < 1 || N < 1 || K < 1 || !A_hi || !B_hi || !D || ldd < N || lda < K || ldb < K ||
        (nsplit != 1 && nsplit != 3) || (sym && M != N) || (H && !coef))
        return CPA_ERR_INVALID_ARG;
    if (!sym && (C || C2 || H || Dhi || Dlo)) return CPA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TcOperand a, b;
    a.hi = (const __nv_bfloat16 *)A_hi; a.lo = (const __nv_bfloat16 *)A_lo; a.ld = lda; a.rows = M;
    b.hi = (const __nv_bfloat16 *)B_hi; b.lo = (const __nv_bfloat16 *)B_lo; b.ld = ldb; b.rows = N;
    Epilogue e;
    e.D = D;
    e.ldd = ldd;
    e.s_acc = s_acc;
    e.C = C;
    e.ldc = ldd;
    e.s_c = s_c;
    e.C2 = C2;
    e.ldc2 = ldd;
    e.s_c2 = s_c2;
    e.diag = diag;
    e.H = H;
    e.ldh = ldd;
    e.coef = coef;
    e.k = k;
    e.Dhi = (__nv_bfloat16 *)Dhi;
    e.Dlo = (__nv_bfloat16 *)Dlo;
    e.ldb = ldh;
    e.symmetric_upper = sym ? 1 : 0;
    cudaError_t r = gemm_tc(M, N, K, a, b, nsplit, e, (cudaStream_t)stream, sms);
    if (r == cudaErrorInvalidValue) return CPA_ERR_INVALID_ARG;
    if (r != cudaSuccess) return cuda_fail(r, "gemm_tc");
    return CPA_OK;
}

cpa_status cpa_kernel_split_bf16(const float *X, int rows, int cols, int64_t ldx, int transpose, void *hi, void *lo,
                                 int64_t ldo, void *stream) {
    if (!X || !hi || rows < 1 || cols < 1 || ldx < cols || ldo < (transpose ? rows : cols))
        return CPA_ERR_INVALID_ARG;
    CK(split_bf16(X, rows, cols, ldx, transpose != 0, (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo, ldo,
                  (cudaStream_t)stream));
    return CPA_OK;
}

cpa_status cpa_kernel_topk_eps(const float *Phi, int p, int64_t ld, long long k, float *eps_host, void *stream) {
    if (!Phi || !eps_host || p < 1 || ld < p || k < 1 || k > (long long)p * (long long)p) return CPA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return CPA_ERR_CUDA;
    char *scratch = nullptr;
    const size_t cbytes = (size_t)kTopkCounts * sizeof(unsigned long long);
    if (cudaMalloc(&scratch, cbytes + 64) != cudaSuccess) {
        cudaGetLastError();
        return CPA_ERR_NO_MEMORY;
    }
    unsigned int *bar = reinterpret_cast<unsigned int *>(scratch + cbytes);
    int *err = reinterpret_cast<int *>(scratch + cbytes + 16);
    float *eps = reinterpret_cast<float *>(scratch + cbytes + 32);
    int err_h = 0;
    cudaError_t e = topk_eps(Phi, p, ld, k, reinterpret_cast<unsigned long long *>(scratch), bar, err, eps, st, sms);
    if (e == cudaSuccess) e = cudaMemcpyAsync(eps_host, eps, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CPA_ERR_CUDA;
    }
    return err_h ? (cpa_status)err_h : CPA_OK;
}

// A sequence of host matrices through cpa_svt with the copies overlapped:
// slot i % 2 holds matrix i on the device.  The H2D copy of matrix i + 1
// (stream h2d) runs while matrix i is shrunk (the caller's stream) and the
// D2H copy of matrix i (stream d2h) runs while matrix i + 1 is; events
// order slot reuse.  The caller's stream waits for the last D2H copy.
cpa_status cpa_svt_host(cpa_handle h, int count, const float *const *hX, int64_t m, int64_t n, int64_t ldx,
                        const cpa_shrink *sh, int L, double lambda_max, int prec, const cpa_sparsify *sp,
                        float *const *hY, int64_t ldy, void *stream) {
    if (!h || count < 0 || (count > 0 && (!hX || !hY)) || m < 1 || n < 1 || ldx < n || ldy < n)
        return CPA_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!hX[i] || !hY[i]) return CPA_ERR_INVALID_ARG;
    if (count == 0) return CPA_OK;
    cpa_status r;
    if ((r = set_device(h)) != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t mat = sizeof(float) * (size_t)(m * n);
    if (h->stage_bytes < 4 * mat) {
        if (h->stage) {
            CK(cudaStreamSynchronize(st));
            if (h->h2d) CK(cudaStreamSynchronize(h->h2d));
            if (h->d2h) CK(cudaStreamSynchronize(h->d2h));
            cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
        }
        if (cudaMalloc(&h->stage, 4 * mat) != cudaSuccess) return CPA_ERR_NO_MEMORY;
        h->stage_bytes = 4 * mat;
    }
    if (!h->h2d) {
        CK(cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(cudaEventCreateWithFlags(&h->in_ready[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->computed[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->out_done[i], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming));
    }
    float *Xd[2] = {h->stage, h->stage + m * n}, *Yd[2] = {h->stage + 2 * m * n, h->stage + 3 * m * n};
    // earlier work on the caller's stream (and an earlier call's copies) first
    CK(cudaEventRecord(h->start, st));
    CK(cudaStreamWaitEvent(h->h2d, h->start, 0));
    CK(cudaStreamWaitEvent(h->d2h, h->start, 0));
    auto h2d = [&](int i) -> cudaError_t {
        const int sl = i & 1;
        if (i >= 2) {
            cudaError_t e = cudaStreamWaitEvent(h->h2d, h->computed[sl], 0);   // matrix i-2 no longer read
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaMemcpy2DAsync(Xd[sl], sizeof(float) * n, hX[i], sizeof(float) * ldx, sizeof(float) * n,
                                          m, cudaMemcpyHostToDevice, h->h2d);
        if (e != cudaSuccess) return e;
        return cudaEventRecord(h->in_ready[sl], h->h2d);
    };
    CK(h2d(0));
    for (int i = 0; i < count; ++i) {
        const int sl = i & 1;
        if (i + 1 < count) CK(h2d(i + 1));
        CK(cudaStreamWaitEvent(st, h->in_ready[sl], 0));
        if (i >= 2) CK(cudaStreamWaitEvent(st, h->out_done[sl], 0));   // Y slot copied out
        if ((r = cpa_svt(h, Xd[sl], m, n, n, sh, L, lambda_max, prec, sp, Yd[sl], n, stream)) != CPA_OK) return r;
        CK(cudaEventRecord(h->computed[sl], st));
        CK(cudaStreamWaitEvent(h->d2h, h->computed[sl], 0));
        CK(cudaMemcpy2DAsync(hY[i], sizeof(float) * ldy, Yd[sl], sizeof(float) * n, sizeof(float) * n, m,
                             cudaMemcpyDeviceToHost, h->d2h));
        CK(cudaEventRecord(h->out_done[sl], h->d2h));
    }
    CK(cudaStreamWaitEvent(st, h->out_done[(count - 1) & 1], 0));
    if (count >= 2) CK(cudaStreamWaitEvent(st, h->out_done[count & 1], 0));
    return CPA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Pointer-form batches: patch-sized members (min(m, n) <= 64, max(m, n) <=
// 128, L within the batched kernel's limit) in one persistent launch, the
// others through the single-matrix path one after another on the stream
// (largest first, so the workspace is sized once).

namespace {


cpa_status check_members(int count, const float *const *dX, const int64_t *m, const int64_t *n, const int64_t *ldx,
                         const cpa_shrink *s, int s_count, float *const *dY, const int64_t *ldy) {
    if (count < 0 || (count > 0 && (!dX || !m || !n || !ldx || !s || !dY || !ldy)) ||
        (s_count != 1 && s_count != count))
        return CPA_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (validate_matrix(dX[i], m[i], n[i], ldx[i]) != CPA_OK || !dY[i] || ldy[i] < n[i])
            return CPA_ERR_INVALID_ARG;
        if (check_shrink(&s[s_count > 1 ? i : 0]) != CPA_OK) return CPA_ERR_INVALID_ARG;
    }
    return CPA_OK;
}

cpa_status ensure_pplan(cpa_ctx *h) {
    if (!h->pplan) h->pplan = ptr_plan_create(h->device, h->num_sms);
    if (!h->pplan_tc) h->pplan_tc = ptr_plan_create(h->device, h->num_sms);
    return h->pplan && h->pplan_tc ? CPA_OK : CPA_ERR_NO_MEMORY;
}

// The member class of the batched launch: 1 for the mma.sync kernel (p <=
// 64, q <= 128; measured faster there, two CTAs per SM), 2 for the tcgen05
// kernel (p <= 128, q <= 4096, tensor-core precisions), 0 for the
// single-matrix path.
int member_class(int64_t m, int64_t n, int L, int prec) {
    const int64_t p = std::min(m, n), q = std::max(m, n);
    if (L > batched_max_terms()) return 0;
    if (p <= 64 && q <= 128) return 1;
    if (prec != CPA_FP32 && p <= kTcBatchP && q <= kTcBatchQ) return 2;
    return 0;
}

// The members `order` (largest first) through fn(handle, k, stream): on the
// caller's handle and stream when h->nstreams is 1 or there is one member,
// else round-robin over sub-handles, each on its own stream forked from the
// caller's stream and joined back into it.
template <class F>
cpa_status run_members(cpa_ctx *h, const std::vector<int> &order, cudaStream_t st, F fn) {
    const int S = std::min<int>(h->nstreams, (int)order.size());
    const int sms = h->member_sms > 0 ? std::min(h->member_sms, h->num_sms) : h->num_sms;
    if (S <= 1 && sms == h->num_sms) {
        for (size_t k = 0; k < order.size(); ++k) {
            cpa_status r = fn(h, (int)k, st);
            if (r != CPA_OK) return r;
        }
        return CPA_OK;
    }
    for (int j = 0; j < S; ++j) {
        if (!h->sub[j]) {
            cpa_status r = cpa_create(&h->sub[j], h->device);
            if (r != CPA_OK) return r;
            CK(cudaStreamCreateWithFlags(&h->sub_st[j], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&h->sub_ev[j], cudaEventDisableTiming));
        }
        h->sub[j]->series = h->series;
        h->sub[j]->num_sms = sms;
        h->sub[j]->profiling = h->profiling;
        h->sub[j]->wait = h->wait;
        h->sub[j]->sparse_skip = h->sparse_skip;
        h->sub[j]->sparse_compact = h->sparse_compact;
    }
    if (!h->fork_ev) CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    CK(cudaEventRecord(h->fork_ev, st));
    for (int j = 0; j < S; ++j) CK(cudaStreamWaitEvent(h->sub_st[j], h->fork_ev, 0));
    cpa_status r = CPA_OK;
    for (size_t k = 0; k < order.size() && r == CPA_OK; ++k) r = fn(h->sub[k % S], (int)k, h->sub_st[k % S]);
    for (int j = 0; j < S; ++j) {
        CK(cudaEventRecord(h->sub_ev[j], h->sub_st[j]));
        CK(cudaStreamWaitEvent(st, h->sub_ev[j], 0));
    }
    return r;
}

std::vector<int> by_size_desc(const std::vector<int> &idx, const int64_t *m, const int64_t *n) {
    std::vector<int> v = idx;
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
        const int64_t pa = std::min(m[a], n[a]), pb = std::min(m[b], n[b]);
        return pa != pb ? pa > pb : std::max(m[a], n[a]) > std::max(m[b], n[b]);
    });
    return v;
}

}  // namespace

extern "C" {

cpa_status cpa_svt_batched(cpa_handle h, int count, const float *const *dX, const int64_t *m, const int64_t *n,
                           const int64_t *ldx, const cpa_shrink *s, int s_count, const int *L, int L0,
                           const double *lambda, int prec, float *const *dY, const int64_t *ldy, void *stream) {
    if (!h) return CPA_ERR_INVALID_ARG;
    cpa_status r = check_members(count, dX, m, n, ldx, s, s_count, dY, ldy);
    if (r != CPA_OK) return r;
    if (prec < CPA_FP32 || prec > CPA_BF16X3) return CPA_ERR_INVALID_ARG;
    if (prec == CPA_TF32 || (prec != CPA_FP32 && h->cc < 100)) return CPA_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        const int Li = L ? L[i] : L0;
        if (Li < 1 || Li > kMaxTerms || (lambda && !(std::isfinite(lambda[i]))))
            return CPA_ERR_INVALID_ARG;
    }
    if (count == 0) return CPA_OK;
    if ((r = set_device(h)) != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> cls[3];
    for (int i = 0; i < count; ++i) cls[member_class(m[i], n[i], L ? L[i] : L0, prec)].push_back(i);
    for (int c = 1; c <= 2; ++c) {
        const std::vector<int> &small = cls[c];
        if (small.empty()) continue;
        if ((r = ensure_pplan(h)) != CPA_OK) return r;
        std::vector<PtrItem> items(small.size());
        std::vector<double> lam(small.size());
        bool all_given = lambda != nullptr;
        for (size_t k = 0; k < small.size(); ++k) {
            const int i = small[k];
            items[k] = PtrItem{dX[i], dY[i], ldx[i], ldy[i], (int)m[i], (int)n[i], L ? L[i] : L0,
                               to_params(&s[s_count > 1 ? i : 0])};
            if (lambda) {
                lam[k] = lambda[i];
                if (!(lambda[i] > 0.0)) all_given = false;
            }
        }
        // the batched kernel takes bounds for all members or none
        if ((r = ptr_plan_run(c == 1 ? h->pplan : h->pplan_tc, (int)small.size(), items.data(),
                              all_given ? lam.data() : nullptr, prec, nullptr, nullptr, st,
                              c == 1 ? CPA_BATCH_MMA_SYNC : CPA_BATCH_TCGEN05)) != CPA_OK)
            return r;
    }
    const std::vector<int> &big = cls[0];
    const std::vector<int> order = by_size_desc(big, m, n);
    return run_members(h, order, st, [&](cpa_ctx *hh, int k, cudaStream_t sk) {
        const int i = order[k];
        return svt_impl(hh, dX[i], m[i], n[i], ldx[i], &s[s_count > 1 ? i : 0], L ? L[i] : L0,
                        lambda ? lambda[i] : 0.0, prec, nullptr, dY[i], ldy[i], sk, nullptr);
    });
}

cpa_status cpa_serve_learned(cpa_handle h, cpa_mlp net, int count, const float *const *dX, const int64_t *m,
                             const int64_t *n, const int64_t *ldx, const cpa_shrink *s, int s_count,
                             const cpa_learn_rule *rule, int prec, float *const *dY, const int64_t *ldy,
                             void *stream) {
    if (!h || !net || !rule) return CPA_ERR_INVALID_ARG;
    cpa_status r = check_members(count, dX, m, n, ldx, s, s_count, dY, ldy);
    if (r != CPA_OK) return r;
    const cpa_learn_rule &ru = *rule;
    if (!(ru.L_scale > 0.0) || !std::isfinite(ru.L_scale) || !(ru.margin >= 0.0) || !std::isfinite(ru.margin) ||
        ru.L_min < 1 || ru.L_max < ru.L_min || ru.L_max > kMaxTerms || ru.L_fallback < 1 || ru.L_fallback > ru.L_max)
        return CPA_ERR_INVALID_ARG;
    if (prec < CPA_FP32 || prec > CPA_BF16X3 || prec == CPA_TF32) return CPA_ERR_UNSUPPORTED;
    int dims[4], dev = -1;
    const float *P = mlp_device_params(net, dims, &dev);
    if (!P || dims[0] != 12 || dims[1] != 64 || dims[2] != 64 || dims[3] != 2 || dev != h->device)
        return CPA_ERR_INVALID_ARG;
    if (h->series != CPA_SERIES_FORWARD) return CPA_ERR_UNSUPPORTED;
    if ((r = set_device(h)) != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    h->serve_small.clear();
    h->serve_mid.clear();
    h->serve_big.clear();
    for (int i = 0; i < count; ++i) {
        const int c = member_class(m[i], n[i], 1, prec);
        (c == 1 ? h->serve_small : c == 2 ? h->serve_mid : h->serve_big).push_back(i);
    }
    for (int c = 1; c <= 2; ++c) {
        const std::vector<int> &grp = c == 1 ? h->serve_small : h->serve_mid;
        if (grp.empty()) continue;
        if ((r = ensure_pplan(h)) != CPA_OK) return r;
        std::vector<PtrItem> items(grp.size());
        for (size_t k = 0; k < items.size(); ++k) {
            const int i = grp[k];
            items[k] = PtrItem{dX[i], dY[i], ldx[i], ldy[i], (int)m[i], (int)n[i], 1,
                               to_params(&s[s_count > 1 ? i : 0])};
        }
        if ((r = ptr_plan_run(c == 1 ? h->pplan : h->pplan_tc, (int)items.size(), items.data(), nullptr, prec, P,
                              rule, st, c == 1 ? CPA_BATCH_MMA_SYNC : CPA_BATCH_TCGEN05)) != CPA_OK)
            return r;
    }
    const int nb = (int)h->serve_big.size();
    if (nb > h->big_cap) {
        CK(cudaStreamSynchronize(st));
        if (h->d_big_L) cudaFree(h->d_big_L);
        if (h->d_big_lam) cudaFree(h->d_big_lam);
        h->d_big_L = nullptr;
        h->d_big_lam = nullptr;
        h->big_cap = 0;
        if (cudaMalloc(&h->d_big_L, sizeof(int) * 2 * nb) != cudaSuccess ||
            cudaMalloc(&h->d_big_lam, sizeof(double) * nb) != cudaSuccess) {
            cudaGetLastError();
            return CPA_ERR_NO_MEMORY;
        }
        h->big_cap = nb;
    }
    h->serve_big = by_size_desc(h->serve_big, m, n);
    LearnCall lc{P, ru};
    r = run_members(h, h->serve_big, st, [&](cpa_ctx *hh, int k, cudaStream_t sk) -> cpa_status {
        const int i = h->serve_big[k];
        cpa_status q = svt_impl(hh, dX[i], m[i], n[i], ldx[i], &s[s_count > 1 ? i : 0], ru.L_max, 0.0, prec,
                                nullptr, dY[i], ldy[i], sk, &lc);
        if (q != CPA_OK) return q;
        // keep this member's choice: the next call reuses the workspace
        CK(cudaMemcpyAsync(h->d_big_L + 2 * k, hh->d_L, 2 * sizeof(int), cudaMemcpyDeviceToDevice, sk));
        CK(cudaMemcpyAsync(h->d_big_lam + k, hh->d_out + 3, sizeof(double), cudaMemcpyDeviceToDevice, sk));
        return CPA_OK;
    });
    h->have_learn = false;
    return r;
}

cpa_status cpa_serve_read(cpa_handle h, int count, int *host_L, double *host_lambda, int *host_fallbacks,
                          void *stream) {
    if (!h || count != (int)(h->serve_small.size() + h->serve_mid.size() + h->serve_big.size()))
        return CPA_ERR_INVALID_ARG;
    cpa_status r = set_device(h);
    if (r != CPA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = (int)h->serve_small.size(), nm = (int)h->serve_mid.size(), nb = (int)h->serve_big.size();
    std::vector<int> sL(ns), mL(nm), bL(2 * nb);
    std::vector<double> sl(ns), ml(nm), bl(nb);
    int nfb_small = 0, nfb_mid = 0;
    if (ns) {
        CK(cudaMemcpyAsync(sL.data(), ptr_plan_orders(h->pplan), sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(sl.data(), ptr_plan_lambdas(h->pplan), sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&nfb_small, ptr_plan_fallbacks(h->pplan), sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    if (nm) {
        CK(cudaMemcpyAsync(mL.data(), ptr_plan_orders(h->pplan_tc), sizeof(int) * nm, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ml.data(), ptr_plan_lambdas(h->pplan_tc), sizeof(double) * nm, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaMemcpyAsync(&nfb_mid, ptr_plan_fallbacks(h->pplan_tc), sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    if (nb) {
        CK(cudaMemcpyAsync(bL.data(), h->d_big_L, sizeof(int) * 2 * nb, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(bl.data(), h->d_big_lam, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    int nfb = nfb_small + nfb_mid;
    for (int k = 0; k < ns; ++k) {
        if (host_L) host_L[h->serve_small[k]] = sL[k];
        if (host_lambda) host_lambda[h->serve_small[k]] = sl[k];
    }
    for (int k = 0; k < nm; ++k) {
        if (host_L) host_L[h->serve_mid[k]] = mL[k];
        if (host_lambda) host_lambda[h->serve_mid[k]] = ml[k];
    }
    for (int k = 0; k < nb; ++k) {
        if (host_L) host_L[h->serve_big[k]] = bL[2 * k];
        if (host_lambda) host_lambda[h->serve_big[k]] = bl[k];
        nfb += bL[2 * k + 1];
    }
    if (host_fallbacks) *host_fallbacks = nfb;
    return CPA_OK;
}

}  // extern "C"
