// Context helpers shared by all stages.
#include <stdarg.h>

#include "common.cuh"

namespace dgec {

dgec_status set_err(Ctx *c, dgec_status s, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
        va_end(ap);
    }
    return s;
}

dgec_status read_counters(Ctx *c, const int64_t *d, int n, int64_t *host) {
    CU_TRY(c, cudaMemcpyAsync(c->h_pinned, d, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(c, cudaStreamSynchronize(c->stream));
    memcpy(host, c->h_pinned, sizeof(int64_t) * n);
    return DGEC_OK;
}

}  // namespace dgec
