// C ABI of the dgec library (include/dgec.h): validation, workspace layout,
// and the Alg. 4 pipeline over the stage kernels.
#include <stdlib.h>

#include <algorithm>

#include "stages.cuh"

using namespace dgec;

struct dgec_ctx {
    Ctx c;
};

namespace {

// Workspace = outputs (kept) followed by one scratch region that every
// stage reuses in turn (sized for the largest stage).
struct Layout {
    Csr csr;
    Skel skel;
    Msf msf;
    Dendro den;
    Condensed cond;
    void *scratch = nullptr;
    size_t total = 0;
};

Problem make_problem(int64_t E, int32_t V, const dgec_params *prm) {
    Problem p;
    p.src = nullptr;
    p.dst = nullptr;
    p.t = nullptr;
    p.E = E;
    p.V = V;
    p.k = prm ? prm->k : 1;
    p.M = prm ? prm->min_cluster_size : 2;
    return p;
}

Layout plan(void *base, const Problem &p) {
    Layout L;
    Arena a(base, SIZE_MAX);
    plan_csr(a, p, L.csr);
    plan_skel(a, p, L.skel);
    plan_msf(a, p, L.msf);
    plan_dendro(a, p, L.den);
    plan_condensed(a, p, L.cond);
    size_t scr = std::max({csr_scratch_bytes(p), skel_scratch_bytes(p), msf_scratch_bytes(p),
                           dendro_scratch_bytes(p), condense_scratch_bytes(p)});
    L.scratch = a.take<char>(scr);
    L.total = a.off + 256;
    return L;
}

dgec_status check_args(Ctx *c, int64_t E, int32_t V, const dgec_params *prm) {
    if (!prm) return set_err(c, DGEC_ERR_INVALID_ARG, "params is null");
    if (E < 0 || V < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "negative size");
    if (E >= (int64_t(1) << 30)) return set_err(c, DGEC_ERR_TOO_LARGE, "n_edges must be < 2^30");
    if (prm->k < 1 || prm->k > 16) return set_err(c, DGEC_ERR_INVALID_ARG, "k must be in [1, 16]");
    if (prm->min_cluster_size < 2) return set_err(c, DGEC_ERR_INVALID_ARG, "min_cluster_size must be >= 2");
    if (prm->flags != 0) return set_err(c, DGEC_ERR_INVALID_ARG, "flags must be 0");
    if (E > 0 && V == 0) return set_err(c, DGEC_ERR_VERTEX_RANGE, "edges but no vertices");
    return DGEC_OK;
}

dgec_status run_pipeline(Ctx *c, Problem &p, Layout &L, dgec_result *out) {
    DG_TRY(stage_csr(c, p, L.csr, L.scratch));
    DG_TRY(stage_skeleton(c, p, L.csr, L.skel, L.scratch));
    DG_TRY(stage_msf(c, p, L.csr, L.skel, L.msf, L.scratch));
    DG_TRY(stage_dendro(c, p, L.csr, L.msf, L.den, L.scratch));
    DG_TRY(stage_condense(c, p, L.msf, L.den, L.cond, L.scratch));
    CU_TRY(c, cudaStreamSynchronize(c->stream));
    CU_TRY(c, cudaGetLastError());
    kt_collect(c);
    out->out_off = L.csr.out_off;
    out->in_off = L.csr.in_off;
    out->out_t = L.csr.out_t;
    out->in_t = L.csr.in_t;
    out->out_id = L.csr.out_id;
    out->in_id = L.csr.in_id;
    out->sk_u = L.skel.u;
    out->sk_v = L.skel.v;
    out->sk_w = L.skel.w;
    out->knn_id = L.skel.knn;
    out->core = L.skel.core;
    out->mst_u = L.msf.u;
    out->mst_v = L.msf.v;
    out->mst_w = L.msf.w;
    out->link_a = L.den.a;
    out->link_b = L.den.b;
    out->link_size = L.den.size;
    out->fall_cluster = L.cond.fall_cluster;
    out->fall_lambda = L.cond.fall_lambda;
    out->cl_id = L.cond.cl_id;
    out->cl_parent = L.cond.cl_parent;
    out->cl_birth = L.cond.cl_birth;
    out->cl_death = L.cond.cl_death;
    out->cl_stab_hi = L.cond.cl_stab_hi;
    out->cl_stab_lo = L.cond.cl_stab_lo;
    out->cl_size = L.cond.cl_size;
    out->cl_selected = L.cond.cl_selected;
    out->labels = L.cond.labels;
    out->n_skeleton = L.skel.n;
    out->n_mst = L.msf.n;
    out->n_condensed = L.cond.n_cl;
    out->n_clusters = L.cond.n_clusters;
    return DGEC_OK;
}

}  // namespace

extern "C" {

dgec_status dgec_create(dgec_ctx **out, int device) {
    if (!out) return DGEC_ERR_INVALID_ARG;
    *out = nullptr;
    dgec_ctx *x = new (std::nothrow) dgec_ctx();
    if (!x) return DGEC_ERR_OOM;
    Ctx *c = &x->c;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_pinned, 4096);
    c->kt = new (std::nothrow) KernelTimer();
    if (e != cudaSuccess) {
        delete x;
        return DGEC_ERR_CUDA;
    }
    *out = x;
    return DGEC_OK;
}

dgec_status dgec_destroy(dgec_ctx *x) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    if (x->c.h_pinned) cudaFreeHost(x->c.h_pinned);
    if (x->c.kt) {
        if (x->c.kt->ev) {
            for (int i = 0; i < 2 * kMaxTimed; i++)
                if (x->c.kt->ev[i]) cudaEventDestroy(x->c.kt->ev[i]);
            free(x->c.kt->ev);
        }
        delete x->c.kt;
    }
    delete x;
    return DGEC_OK;
}

const char *dgec_last_error(const dgec_ctx *x) { return x ? x->c.msg : "null context"; }

const char *dgec_status_string(dgec_status s) {
    switch (s) {
        case DGEC_OK: return "ok";
        case DGEC_ERR_INVALID_ARG: return "invalid argument";
        case DGEC_ERR_VERTEX_RANGE: return "vertex id out of range";
        case DGEC_ERR_SELF_LOOP: return "self loop";
        case DGEC_ERR_TOO_LARGE: return "input too large";
        case DGEC_ERR_OOM: return "workspace too small";
        case DGEC_ERR_CUDA: return "CUDA error";
        case DGEC_ERR_TIMEOUT: return "iteration bound exceeded";
        default: return "internal error";
    }
}

int64_t dgec_last_launch_count(const dgec_ctx *x) { return x ? x->c.launches : -1; }

dgec_status dgec_set_kernel_timing(dgec_ctx *x, int mode, const char *name) {
    if (!x || !x->c.kt || mode < 0 || mode > 2 || (mode == 1 && !name))
        return DGEC_ERR_INVALID_ARG;
    KernelTimer *k = x->c.kt;
    k->mode = mode;
    snprintf(k->only, sizeof(k->only), "%s", mode == 1 ? name : "");
    k->used = 0;
    k->n_names = 0;
    return DGEC_OK;
}

dgec_status dgec_kernel_timing(dgec_ctx *x, int i, const char **name, double *total_ms,
                               int64_t *launches) {
    if (!x || !x->c.kt) return DGEC_ERR_INVALID_ARG;
    kt_collect(&x->c);
    KernelTimer *k = x->c.kt;
    if (i < 0 || i >= k->n_names) return DGEC_ERR_INVALID_ARG;
    if (name) *name = k->names[i];
    if (total_ms) *total_ms = k->ms[i];
    if (launches) *launches = k->count[i];
    return DGEC_OK;
}

dgec_status dgec_workspace_size(int64_t n_edges, int32_t n_vertices, const dgec_params *params,
                                size_t *bytes) {
    if (!bytes) return DGEC_ERR_INVALID_ARG;
    dgec_status s = check_args(nullptr, n_edges, n_vertices, params);
    if (s != DGEC_OK) return s;
    Problem p = make_problem(n_edges, n_vertices, params);
    *bytes = plan(nullptr, p).total;
    return DGEC_OK;
}

dgec_status dgec_run(dgec_ctx *x, const int32_t *d_src, const int32_t *d_dst, const int64_t *d_t,
                     int64_t n_edges, int32_t n_vertices, const dgec_params *params, void *d_ws,
                     size_t ws_bytes, void *stream, dgec_result *out) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    c->launches = 0;
    DG_TRY(check_args(c, n_edges, n_vertices, params));
    if (!out) return set_err(c, DGEC_ERR_INVALID_ARG, "out is null");
    if (n_edges > 0 && (!d_src || !d_dst || !d_t)) return set_err(c, DGEC_ERR_INVALID_ARG, "null input");
    if (!d_ws || ((uintptr_t)d_ws & 255)) return set_err(c, DGEC_ERR_INVALID_ARG, "workspace null or not 256-byte aligned");
    CU_TRY(c, cudaSetDevice(c->device));
    c->stream = (cudaStream_t)stream;
    Problem p = make_problem(n_edges, n_vertices, params);
    p.src = d_src;
    p.dst = d_dst;
    p.t = d_t;
    size_t need = plan(nullptr, p).total;
    if (ws_bytes < need)
        return set_err(c, DGEC_ERR_OOM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    Layout L = plan(d_ws, p);
    memset(out, 0, sizeof(*out));
    return run_pipeline(c, p, L, out);
}

dgec_status dgec_run_host(dgec_ctx *x, const int32_t *h_src, const int32_t *h_dst, const int64_t *h_t,
                          int64_t n_edges, int32_t n_vertices, const dgec_params *params, void *d_ws,
                          size_t ws_bytes, void *stream, int32_t *h_labels, int32_t *h_n_clusters) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    DG_TRY(check_args(c, n_edges, n_vertices, params));
    if (n_edges > 0 && (!h_src || !h_dst || !h_t || !h_labels))
        return set_err(c, DGEC_ERR_INVALID_ARG, "null host pointer");
    if (!d_ws || ((uintptr_t)d_ws & 255)) return set_err(c, DGEC_ERR_INVALID_ARG, "workspace null or not 256-byte aligned");
    CU_TRY(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    // inputs go at the front of the workspace, the pipeline after them
    Arena a(d_ws, ws_bytes);
    int32_t *d_src = a.take<int32_t>(n_edges);
    int32_t *d_dst = a.take<int32_t>(n_edges);
    int64_t *d_t = a.take<int64_t>(n_edges);
    size_t head = (a.off + 255) & ~(size_t)255;
    if (head > ws_bytes) return set_err(c, DGEC_ERR_OOM, "workspace too small for the inputs");
    if (n_edges > 0) {
        CU_TRY(c, cudaMemcpyAsync(d_src, h_src, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, st));
        CU_TRY(c, cudaMemcpyAsync(d_dst, h_dst, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, st));
        CU_TRY(c, cudaMemcpyAsync(d_t, h_t, sizeof(int64_t) * n_edges, cudaMemcpyHostToDevice, st));
    }
    dgec_result r;
    DG_TRY(dgec_run(x, d_src, d_dst, d_t, n_edges, n_vertices, params, (char *)d_ws + head,
                    ws_bytes - head, stream, &r));
    if (n_edges > 0) {
        CU_TRY(c, cudaMemcpyAsync(h_labels, r.labels, sizeof(int32_t) * n_edges, cudaMemcpyDeviceToHost, st));
        CU_TRY(c, cudaStreamSynchronize(st));
    }
    if (h_n_clusters) *h_n_clusters = r.n_clusters;
    return DGEC_OK;
}

}  // extern "C"
