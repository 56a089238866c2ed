// Context helpers shared by all stages.
#include <stdarg.h>

#include "common.cuh"

namespace dgec {

thread_local int64_t tl_stream_ctas = 65536;

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

int kt_begin(Ctx *c, const char *name) {
    KernelTimer *k = c->kt;
    if (!k || k->mode == 0) return -1;
    if (k->mode == 1 && strcmp(k->only, name) != 0) return -1;
    if (k->mode == 3 && strncmp(k->only, name, strlen(k->only)) != 0) return -1;
    if (k->used >= kMaxTimed) return -1;
    if (!k->ev) {
        k->ev = (cudaEvent_t *)calloc(2 * kMaxTimed, sizeof(cudaEvent_t));
        if (!k->ev) return -1;
    }
    int slot = k->used++;
    int id = -1;
    for (int i = 0; i < k->n_names; i++)
        if (k->names[i] == name || strcmp(k->names[i], name) == 0) id = i;
    if (id < 0 && k->n_names < kMaxNames) {
        id = k->n_names++;
        k->names[id] = name;
        k->ms[id] = 0;
        k->count[id] = 0;
    }
    k->name_of[slot] = id;
    for (int e = 0; e < 2; e++)
        if (!k->ev[2 * slot + e]) cudaEventCreate(&k->ev[2 * slot + e]);
    cudaEventRecord(k->ev[2 * slot], c->stream);
    return slot;
}

void kt_end(Ctx *c, int slot) {
    if (slot < 0) return;
    cudaEventRecord(c->kt->ev[2 * slot + 1], c->stream);
}

// Fold recorded event pairs into per-name totals (synchronises on them).
void kt_collect(Ctx *c) {
    KernelTimer *k = c->kt;
    if (!k) return;
    for (int s = 0; s < k->used; s++) {
        float ms = 0;
        cudaEventSynchronize(k->ev[2 * s + 1]);
        cudaEventElapsedTime(&ms, k->ev[2 * s], k->ev[2 * s + 1]);
        int id = k->name_of[s];
        if (id >= 0) {
            k->ms[id] += ms;
            k->count[id] += 1;
        }
    }
    k->used = 0;
}

void stage_start(Ctx *c) {
    StageTimer &t = c->stages;
    t.n = 0;
    if (!t.ev[0] && cudaEventCreate(&t.ev[0]) != cudaSuccess) return;
    cudaEventRecord(t.ev[0], c->stream);
}

void stage_mark(Ctx *c, const char *name) {
    StageTimer &t = c->stages;
    if (!t.ev[0] || t.n >= kMaxStages) return;
    if (!t.ev[t.n + 1] && cudaEventCreate(&t.ev[t.n + 1]) != cudaSuccess) return;
    cudaEventRecord(t.ev[t.n + 1], c->stream);
    t.name[t.n] = name;
    t.n++;
}

// Per-stage milliseconds from consecutive events (synchronises on the last).
void stage_collect(Ctx *c) {
    StageTimer &t = c->stages;
    if (t.n == 0) return;
    cudaEventSynchronize(t.ev[t.n]);
    for (int i = 0; i < t.n; i++) {
        float ms = 0;
        cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]);
        t.ms[i] = ms;
    }
}

}  // namespace dgec
