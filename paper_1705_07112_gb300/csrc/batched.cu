// Batched shrinkage of many small matrices (patch groups).
#include "internal.h"

struct cpa_batch_ctx {
    int count = 0;
};

extern "C" {

cpa_status cpa_batch_create(cpa_handle h, int count, const int64_t *off, const int32_t *m, const int32_t *n,
                            const int32_t *L, int L0, cpa_batch *out) {
    (void)h; (void)count; (void)off; (void)m; (void)n; (void)L; (void)L0;
    if (out) *out = nullptr;
    return CPA_ERR_UNSUPPORTED;
}

cpa_status cpa_batch_destroy(cpa_batch b) {
    delete b;
    return CPA_OK;
}

cpa_status cpa_svt_batched(cpa_handle h, cpa_batch b, const float *dX, const cpa_shrink *s, int s_count,
                           const double *lambda, int iters, int prec, float *dY, void *stream) {
    (void)h; (void)b; (void)dX; (void)s; (void)s_count; (void)lambda; (void)iters; (void)prec; (void)dY;
    (void)stream;
    return CPA_ERR_UNSUPPORTED;
}

const double *cpa_batch_lambdas(cpa_batch b) {
    (void)b;
    return nullptr;
}

}  // extern "C"
