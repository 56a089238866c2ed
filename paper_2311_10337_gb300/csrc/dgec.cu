// C ABI of the dgec library (include/dgec.h): validation, workspace layout,
// and the Alg. 4 pipeline over the stage kernels.
#include <stdlib.h>

#include <algorithm>

#include "levels.cuh"

using namespace dgec;

namespace {

// Workspace = per-graph tables and outputs (kept) followed by one scratch
// region that every stage reuses in turn (sized for the largest stage).
struct Layout {
    int64_t *eoff, *voff, *knn_off;
    int32_t *gk, *gM, *egraph;
    Csr csr;
    Skel skel;
    Skel mrd;  // stage M output (mutual-reachability mode only)
    bool nc = false;  // nearly-causal mode: stage A/B again on negated times, stage N
    int64_t *tneg = nullptr;
    Csr csr2;
    Skel skel2, ncs;
    Msf msf;
    Dendro den;
    Condensed cond;
    int32_t *lmu, *lmv, *lla, *llb;  // batch outputs in each graph's local ids
    void *scratch = nullptr;
    size_t total = 0;
};

// Host-side description of a batch (a plain run is one graph).
struct HostBatch {
    int32_t G;
    const int64_t *eoff;  // [G+1]
    const int32_t *nv;    // [G]
    const int32_t *k;     // [G]
    const int32_t *M;     // [G]
    int64_t dmax = INT64_MAX;  // time cutoff, INT64_MAX = none
    bool mrd = false;          // mutual-reachability mode (one graph only)
    int64_t dnc = 0;           // nearly-causal tolerance (one graph only), 0 = causal
};

Problem make_problem(const HostBatch &hb) {
    Problem p;
    p.src = nullptr;
    p.dst = nullptr;
    p.t = nullptr;
    p.G = hb.G;
    p.E = hb.eoff[hb.G];
    int64_t V = 0;
    int kmax = 1, Mmin = 1 << 30;
    for (int g = 0; g < hb.G; g++) {
        V += hb.nv[g];
        kmax = std::max(kmax, hb.k[g]);
        Mmin = std::min(Mmin, hb.M[g]);
    }
    p.V = V;
    p.k = kmax;
    p.M = Mmin;
    p.dmax = hb.dmax;
    p.mrd = hb.mrd;
    p.dnc = hb.dnc;
    if (p.mrd) p.links_cap = 2 * p.E + p.E * (int64_t)p.k;
    if (p.dnc > 0) p.links_cap = 4 * p.E;
    return p;
}

Layout plan(void *base, const Problem &p) {
    Layout L;
    Arena a(base, SIZE_MAX);
    L.eoff = a.take<int64_t>(p.G + 1);
    L.voff = a.take<int64_t>(p.G + 1);
    L.knn_off = a.take<int64_t>(p.G + 1);
    L.gk = a.take<int32_t>(p.G);
    L.gM = a.take<int32_t>(p.G);
    L.egraph = a.take<int32_t>(p.E);
    plan_csr(a, p, L.csr);
    plan_skel(a, p, L.skel);
    if (p.mrd) plan_mrd(a, p, L.mrd);
    if (p.dnc > 0) {
        L.nc = true;
        L.tneg = a.take<int64_t>(p.E);
        plan_csr(a, p, L.csr2);
        plan_skel(a, p, L.skel2);
        plan_nc(a, p, L.ncs);
    }
    plan_msf(a, p, L.msf);
    plan_dendro(a, p, L.den);
    plan_condensed(a, p, L.cond);
    if (p.G > 1) {
        L.lmu = a.take<int32_t>(p.E);
        L.lmv = a.take<int32_t>(p.E);
        L.lla = a.take<int32_t>(p.E);
        L.llb = a.take<int32_t>(p.E);
    } else {
        L.lmu = L.lmv = L.lla = L.llb = nullptr;
    }
    size_t scr = std::max({csr_scratch_bytes(p), skel_scratch_bytes(p), msf_scratch_bytes(p),
                           dendro_scratch_bytes(p), condense_scratch_bytes(p)});
    if (p.mrd) scr = std::max(scr, mrd_scratch_bytes(p));
    if (p.dnc > 0) scr = std::max(scr, nc_scratch_bytes(p));
    L.scratch = a.take<char>(scr);
    L.total = a.off + 256;
    return L;
}

dgec_status check_batch(Ctx *c, const HostBatch &hb) {
    if (hb.G < 1 || !hb.eoff || !hb.nv || !hb.k || !hb.M)
        return set_err(c, DGEC_ERR_INVALID_ARG, "bad batch description");
    if (hb.eoff[0] != 0) return set_err(c, DGEC_ERR_INVALID_ARG, "edge offsets must start at 0");
    int64_t V = 0;
    for (int g = 0; g < hb.G; g++) {
        int64_t Eg = hb.eoff[g + 1] - hb.eoff[g];
        if (Eg < 0 || hb.nv[g] < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "graph %d: negative size", g);
        if (Eg > 0 && hb.nv[g] == 0) return set_err(c, DGEC_ERR_VERTEX_RANGE, "graph %d: edges but no vertices", g);
        if (hb.k[g] < 1 || hb.k[g] > 16) return set_err(c, DGEC_ERR_INVALID_ARG, "k must be in [1, 16]");
        if (hb.M[g] < 2) return set_err(c, DGEC_ERR_INVALID_ARG, "min_cluster_size must be >= 2");
        V += hb.nv[g];
    }
    if (hb.eoff[hb.G] >= (int64_t(1) << 30)) return set_err(c, DGEC_ERR_TOO_LARGE, "total edges must be < 2^30");
    if (V >= (int64_t(1) << 31)) return set_err(c, DGEC_ERR_TOO_LARGE, "total vertices must be < 2^31");
    return DGEC_OK;
}

dgec_status check_params(Ctx *c, const dgec_params *prm) {
    if (!prm) return set_err(c, DGEC_ERR_INVALID_ARG, "params is null");
    if (prm->flags & ~(DGEC_CUTOFF | DGEC_MRD | DGEC_NEARLY_CAUSAL))
        return set_err(c, DGEC_ERR_INVALID_ARG, "unknown flags");
    if ((prm->flags & DGEC_NEARLY_CAUSAL) && prm->delta_nc < 0)
        return set_err(c, DGEC_ERR_INVALID_ARG, "delta_nc must be >= 0");
    if ((prm->flags & DGEC_NEARLY_CAUSAL) && (prm->flags & DGEC_MRD))
        return set_err(c, DGEC_ERR_INVALID_ARG, "the nearly-causal and mutual-reachability modes do not combine");
    if ((prm->flags & DGEC_CUTOFF) && prm->delta_max < 0)
        return set_err(c, DGEC_ERR_INVALID_ARG, "delta_max must be >= 0");
    return DGEC_OK;
}

// batch outputs in local ids: forest ends and dendrogram children
__global__ void k_localize(int64_t n, int64_t E, const int32_t *mu, const int32_t *mv, const int32_t *la,
                           const int32_t *lb, const int32_t *egraph, const int64_t *eoff,
                           const int64_t *goff, int32_t *lmu, int32_t *lmv, int32_t *lla,
                           int32_t *llb) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int g = egraph[mu[s]];
        int64_t e0 = eoff[g], Eg = eoff[g + 1] - e0, m0 = goff[g];
        lmu[s] = (int32_t)(mu[s] - e0);
        lmv[s] = (int32_t)(mv[s] - e0);
        int a = la[s], b = lb[s];
        lla[s] = (int32_t)(a < E ? a - e0 : Eg + (a - E - m0));
        llb[s] = (int32_t)(b < E ? b - e0 : Eg + (b - E - m0));
    }
}

// Per-graph tables, staged through host arrays, one copy each.
dgec_status upload_tables(Ctx *c, const HostBatch &hb, int64_t *eoff, int64_t *voff, int64_t *knn_off,
                          int32_t *gk, int32_t *gM) {
    int G = hb.G;
    int64_t *hv = (int64_t *)malloc(sizeof(int64_t) * (3 * (size_t)(G + 1)));
    if (!hv) return set_err(c, DGEC_ERR_OOM, "host memory");
    int64_t *hvoff = hv, *hknn = hv + (G + 1), *heoff = hv + 2 * (G + 1);
    hvoff[0] = 0;
    hknn[0] = 0;
    for (int g = 0; g < G; g++) {
        heoff[g] = hb.eoff[g];
        hvoff[g + 1] = hvoff[g] + hb.nv[g];
        hknn[g + 1] = hknn[g] + (hb.eoff[g + 1] - hb.eoff[g]) * hb.k[g];
    }
    heoff[G] = hb.eoff[G];
    cudaError_t e1 = cudaMemcpyAsync(eoff, heoff, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(voff, hvoff, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, c->stream);
    cudaError_t e3 = cudaMemcpyAsync(knn_off, hknn, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, c->stream);
    cudaError_t e4 = cudaMemcpyAsync(gk, hb.k, sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream);
    cudaError_t e5 = cudaMemcpyAsync(gM, hb.M, sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream);
    cudaError_t e6 = cudaStreamSynchronize(c->stream);
    free(hv);
    if (e1 || e2 || e3 || e4 || e5 || e6) return set_err(c, DGEC_ERR_CUDA, "copying the batch tables failed");
    return DGEC_OK;
}

dgec_status run_pipeline(Ctx *c, const HostBatch &hb, const int32_t *d_src, const int32_t *d_dst,
                         const int64_t *d_t, void *d_ws, size_t ws_bytes, Layout *out_layout,
                         Problem *out_problem) {
    Problem p = make_problem(hb);
    p.src = d_src;
    p.dst = d_dst;
    p.t = d_t;
    if (p.E > 0 && (!d_src || !d_dst || !d_t)) return set_err(c, DGEC_ERR_INVALID_ARG, "null input");
    if (!d_ws || ((uintptr_t)d_ws & 255))
        return set_err(c, DGEC_ERR_INVALID_ARG, "workspace null or not 256-byte aligned");
    size_t need = plan(nullptr, p).total;
    if (ws_bytes < need) return set_err(c, DGEC_ERR_OOM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    Layout L = plan(d_ws, p);
    DG_TRY(upload_tables(c, hb, L.eoff, L.voff, L.knn_off, L.gk, L.gM));
    p.eoff = L.eoff;
    p.voff = L.voff;
    p.knn_off = L.knn_off;
    p.gk = L.gk;
    p.gM = L.gM;
    p.egraph = L.egraph;
    tl_stream_ctas = c->stream_ctas;
    stage_start(c);
    DG_STAGE("A incidence lists", stage_csr(c, p, L.csr, L.scratch));
    DG_STAGE("B skeleton and kNN", stage_skeleton(c, p, L.csr, L.skel, L.scratch));
    const Skel *forest_in = &L.skel;
    if (p.dnc > 0) {
        DG_STAGE("N negated times", stage_nc_negate(c, p, L.tneg));
        Problem p2 = p;
        p2.t = L.tneg;
        DG_STAGE("A incidence lists", stage_csr(c, p2, L.csr2, L.scratch));
        DG_STAGE("B skeleton and kNN", stage_skeleton(c, p2, L.csr2, L.skel2, L.scratch));
        DG_STAGE("N nearly-causal union", stage_nc(c, p, L.csr, L.skel, L.skel2, L.ncs, L.scratch));
        forest_in = &L.ncs;
    }
    if (p.mrd) {
        DG_STAGE("R mutual-reachability graph", stage_mrd(c, p, L.csr, L.skel, L.mrd, L.scratch));
        forest_in = &L.mrd;
    }
    DG_STAGE("C spanning forest", stage_msf(c, p, L.csr, *forest_in, L.msf, L.scratch));
    DG_STAGE("D1 dendrogram", stage_dendro(c, p, L.csr, L.msf, L.den, L.scratch));
    DG_STAGE("D2 condense and labels", stage_condense(c, p, L.msf, L.den, L.cond, L.scratch));
    if (p.G > 1 && L.msf.n > 0)
        TK(c, "k_localize", k_localize<<<grid_for(L.msf.n, kBlock, kStreamCap), kBlock, 0, c->stream>>>(
                                L.msf.n, p.E, L.msf.u, L.msf.v, L.den.a, L.den.b, p.egraph, p.eoff,
                                L.msf.goff, L.lmu, L.lmv, L.lla, L.llb));
    CU_TRY(c, cudaStreamSynchronize(c->stream));
    CU_TRY(c, cudaGetLastError());
    kt_collect(c);
    stage_collect(c);
    *out_layout = L;
    *out_problem = p;
    return DGEC_OK;
}

void fill_result(const Layout &L, dgec_result *out) {
    out->out_off = L.csr.out_off;
    out->in_off = L.csr.in_off;
    out->out_t = L.csr.out_t;
    out->in_t = L.csr.in_t;
    out->out_id = L.csr.out_id;
    out->in_id = L.csr.in_id;
    out->pos_out = L.csr.pos_out;
    out->pos_in = L.csr.pos_in;
    const Skel &sk = L.nc ? L.ncs : L.skel;
    out->sk_u = sk.u;
    out->sk_v = sk.v;
    out->sk_w = sk.w;
    out->knn_id = sk.knn;
    out->core = sk.core;
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
    out->n_skeleton = sk.n;
    out->n_mst = L.msf.n;
    out->n_condensed = L.cond.n_cl;
    out->n_clusters = L.cond.n_clusters;
}


// ------------------------------------------------- discrete dendrogram run

struct LvLayout {
    int64_t *eoff, *voff, *knn_off;
    int32_t *gk, *gM, *egraph;
    Csr csr;
    Skel skel;
    Levels lv;
    Dendro den;
    Condensed cond;
    void *scratch = nullptr;
    size_t total = 0;
};

LvLayout plan_lv(void *base, const Problem &p, int q, bool dense, bool condense) {
    LvLayout L;
    Arena a(base, SIZE_MAX);
    L.eoff = a.take<int64_t>(2);
    L.voff = a.take<int64_t>(2);
    L.knn_off = a.take<int64_t>(2);
    L.gk = a.take<int32_t>(1);
    L.gM = a.take<int32_t>(1);
    L.egraph = a.take<int32_t>(p.E);
    plan_csr(a, p, L.csr);
    plan_skel(a, p, L.skel);
    plan_levels(a, p, q, dense, L.lv);
    size_t scr = std::max({csr_scratch_bytes(p), skel_scratch_bytes(p), levels_scratch_bytes(p)});
    if (condense) {
        plan_dendro(a, p, L.den);
        plan_condensed(a, p, L.cond);
        scr = std::max({scr, dendro_scratch_bytes(p), condense_scratch_bytes(p)});
    }
    L.scratch = a.take<char>(scr);
    L.total = a.off + 256;
    return L;
}

dgec_status check_levels(Ctx *c, const dgec_levels_params *lp) {
    if (!lp) return set_err(c, DGEC_ERR_INVALID_ARG, "params is null");
    if (lp->n_levels < 1 || lp->n_levels > kMaxLevels)
        return set_err(c, DGEC_ERR_INVALID_ARG, "n_levels must be in [1, %d]", kMaxLevels);
    if (!lp->h_omega) return set_err(c, DGEC_ERR_INVALID_ARG, "thresholds are null");
    for (int i = 0; i < lp->n_levels; i++) {
        if (lp->h_omega[i] < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "threshold %d is negative", i);
        if (i > 0 && lp->h_omega[i] <= lp->h_omega[i - 1])
            return set_err(c, DGEC_ERR_INVALID_ARG, "thresholds must be strictly increasing");
    }
    if (lp->min_cluster_size != 0 && lp->min_cluster_size < 2)
        return set_err(c, DGEC_ERR_INVALID_ARG, "min_cluster_size must be 0 or >= 2");
    if (lp->flags & ~DGEC_LEVELS_DENSE) return set_err(c, DGEC_ERR_INVALID_ARG, "unknown flags");
    return DGEC_OK;
}

// The batch-of-one description the stages expect; k is unused (no kNN).
struct LvDesc {
    int64_t eoff[2];
    int32_t nv, k = 1, M;
    HostBatch hb() const { return HostBatch{1, eoff, &nv, &k, &M}; }
};
LvDesc lv_desc(int64_t E, int32_t V, const dgec_levels_params *lp) {
    LvDesc d;
    d.eoff[0] = 0;
    d.eoff[1] = E;
    d.nv = V;
    d.M = lp->min_cluster_size ? lp->min_cluster_size : 2;
    return d;
}
Problem lv_problem(const LvDesc &d) {
    Problem p = make_problem(d.hb());
    p.knn = false;
    return p;
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
    if (e != cudaSuccess || !c->kt) {
        if (c->h_pinned) cudaFreeHost(c->h_pinned);
        delete c->kt;
        delete x;
        return e != cudaSuccess ? DGEC_ERR_CUDA : DGEC_ERR_OOM;
    }
    *out = x;
    return DGEC_OK;
}

dgec_status dgec_destroy(dgec_ctx *x) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    if (x->c.h_pinned) cudaFreeHost(x->c.h_pinned);
    for (int i = 0; i <= kMaxStages; i++)
        if (x->c.stages.ev[i]) cudaEventDestroy(x->c.stages.ev[i]);
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
        case DGEC_ERR_TIMEOUT: return "iteration bound exceeded or wait timed out";
        case DGEC_ERR_ADMISSION: return "job can never fit a lane";
        default: return "internal error";
    }
}

int64_t dgec_last_launch_count(const dgec_ctx *x) { return x ? x->c.launches : -1; }

dgec_status dgec_set_kernel_timing(dgec_ctx *x, int mode, const char *name) {
    if (!x || !x->c.kt || mode < 0 || mode > 3 || ((mode == 1 || mode == 3) && !name))
        return DGEC_ERR_INVALID_ARG;
    KernelTimer *k = x->c.kt;
    k->mode = mode;
    snprintf(k->only, sizeof(k->only), "%s", (mode == 1 || mode == 3) ? name : "");
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

dgec_status dgec_set_launch_config(dgec_ctx *x, const dgec_launch_config *cfg) {
    if (!x || !cfg) return DGEC_ERR_INVALID_ARG;
    if (cfg->knn_block != 64 && cfg->knn_block != 128 && cfg->knn_block != 256)
        return set_err(&x->c, DGEC_ERR_INVALID_ARG, "knn_block must be 64, 128 or 256");
    if (cfg->stream_ctas < 1 || cfg->stream_ctas > (1 << 20))
        return set_err(&x->c, DGEC_ERR_INVALID_ARG, "stream_ctas must be in [1, 2^20]");
    if (cfg->knn_packed < 0 || cfg->knn_packed > 2)
        return set_err(&x->c, DGEC_ERR_INVALID_ARG, "knn_packed must be 0, 1 or 2");
    x->c.knn_block = cfg->knn_block;
    x->c.stream_ctas = cfg->stream_ctas;
    x->c.knn_packed = cfg->knn_packed;
    return DGEC_OK;
}

dgec_status dgec_get_launch_config(const dgec_ctx *x, dgec_launch_config *cfg) {
    if (!x || !cfg) return DGEC_ERR_INVALID_ARG;
    cfg->knn_block = x->c.knn_block;
    cfg->stream_ctas = (int32_t)x->c.stream_ctas;
    cfg->knn_packed = x->c.knn_packed;
    return DGEC_OK;
}

dgec_status dgec_stage_timing(const dgec_ctx *x, int i, const char **name, double *ms) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    const StageTimer &t = x->c.stages;
    if (i < 0 || i >= t.n) return DGEC_ERR_INVALID_ARG;
    if (name) *name = t.name[i];
    if (ms) *ms = t.ms[i];
    return DGEC_OK;
}

dgec_status dgec_workspace_size(int64_t n_edges, int32_t n_vertices, const dgec_params *params,
                                size_t *bytes) {
    if (!bytes) return DGEC_ERR_INVALID_ARG;
    DG_TRY(check_params(nullptr, params));
    int64_t eoff[2] = {0, n_edges};
    HostBatch hb{1, eoff, &n_vertices, &params->k, &params->min_cluster_size};
    hb.mrd = params->flags & DGEC_MRD;
    if (params->flags & DGEC_NEARLY_CAUSAL) hb.dnc = params->delta_nc;
    if (n_edges < 0) return DGEC_ERR_INVALID_ARG;
    DG_TRY(check_batch(nullptr, hb));
    *bytes = plan(nullptr, make_problem(hb)).total;
    return DGEC_OK;
}

dgec_status dgec_run(dgec_ctx *x, const int32_t *d_src, const int32_t *d_dst, const int64_t *d_t,
                     int64_t n_edges, int32_t n_vertices, const dgec_params *params, void *d_ws,
                     size_t ws_bytes, void *stream, dgec_result *out) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    c->launches = 0;
    DG_TRY(check_params(c, params));
    if (!out) return set_err(c, DGEC_ERR_INVALID_ARG, "out is null");
    if (n_edges < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "negative size");
    int64_t eoff[2] = {0, n_edges};
    HostBatch hb{1, eoff, &n_vertices, &params->k, &params->min_cluster_size};
    if (params->flags & DGEC_CUTOFF) hb.dmax = params->delta_max;
    hb.mrd = params->flags & DGEC_MRD;
    if (params->flags & DGEC_NEARLY_CAUSAL) hb.dnc = params->delta_nc;
    DG_TRY(check_batch(c, hb));
    CU_TRY(c, cudaSetDevice(c->device));
    c->stream = (cudaStream_t)stream;
    Layout L;
    Problem p;
    memset(out, 0, sizeof(*out));
    DG_TRY(run_pipeline(c, hb, d_src, d_dst, d_t, d_ws, ws_bytes, &L, &p));
    fill_result(L, out);
    return DGEC_OK;
}

dgec_status dgec_batch_workspace_size(int32_t n_graphs, const int64_t *h_edge_off,
                                      const int32_t *h_n_vertices, const int32_t *h_k,
                                      const int32_t *h_min_cluster_size, size_t *bytes) {
    if (!bytes) return DGEC_ERR_INVALID_ARG;
    HostBatch hb{n_graphs, h_edge_off, h_n_vertices, h_k, h_min_cluster_size};
    DG_TRY(check_batch(nullptr, hb));
    *bytes = plan(nullptr, make_problem(hb)).total;
    return DGEC_OK;
}

dgec_status dgec_run_batch(dgec_ctx *x, int32_t n_graphs, const int64_t *h_edge_off,
                           const int32_t *h_n_vertices, const int32_t *h_k,
                           const int32_t *h_min_cluster_size, const int32_t *d_src,
                           const int32_t *d_dst, const int64_t *d_t, void *d_ws, size_t ws_bytes,
                           void *stream, dgec_batch_result *out) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    c->launches = 0;
    if (!out) return set_err(c, DGEC_ERR_INVALID_ARG, "out is null");
    HostBatch hb{n_graphs, h_edge_off, h_n_vertices, h_k, h_min_cluster_size};
    DG_TRY(check_batch(c, hb));
    CU_TRY(c, cudaSetDevice(c->device));
    c->stream = (cudaStream_t)stream;
    Layout L;
    Problem p;
    memset(out, 0, sizeof(*out));
    DG_TRY(run_pipeline(c, hb, d_src, d_dst, d_t, d_ws, ws_bytes, &L, &p));
    fill_result(L, &out->global);
    bool local = n_graphs > 1;
    out->labels = L.cond.labels;
    out->knn_id = L.skel.knn;
    out->core = L.skel.core;
    out->mst_u = local ? L.lmu : L.msf.u;
    out->mst_v = local ? L.lmv : L.msf.v;
    out->mst_w = L.msf.w;
    out->link_a = local ? L.lla : L.den.a;
    out->link_b = local ? L.llb : L.den.b;
    out->link_size = L.den.size;
    out->n_clusters = L.cond.gclusters;
    out->mst_off = L.msf.goff;
    out->knn_off = L.knn_off;
    out->total_edges = p.E;
    out->total_mst = L.msf.n;
    out->total_clusters = L.cond.n_clusters;
    return DGEC_OK;
}

dgec_status dgec_run_host(dgec_ctx *x, const int32_t *h_src, const int32_t *h_dst, const int64_t *h_t,
                          int64_t n_edges, int32_t n_vertices, const dgec_params *params, void *d_ws,
                          size_t ws_bytes, void *stream, int32_t *h_labels, int32_t *h_n_clusters) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    DG_TRY(check_params(c, params));
    if (n_edges < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "negative size");
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

dgec_status dgec_levels_workspace_size(int64_t n_edges, int32_t n_vertices, const dgec_levels_params *params,
                                       size_t *bytes) {
    if (!bytes || n_edges < 0) return DGEC_ERR_INVALID_ARG;
    DG_TRY(check_levels(nullptr, params));
    LvDesc d = lv_desc(n_edges, n_vertices, params);
    DG_TRY(check_batch(nullptr, d.hb()));
    *bytes = plan_lv(nullptr, lv_problem(d), params->n_levels, params->flags & DGEC_LEVELS_DENSE,
                     params->min_cluster_size != 0)
                 .total;
    return DGEC_OK;
}

dgec_status dgec_run_levels(dgec_ctx *x, const int32_t *d_src, const int32_t *d_dst, const int64_t *d_t,
                            int64_t n_edges, int32_t n_vertices, const dgec_levels_params *params, void *d_ws,
                            size_t ws_bytes, void *stream, dgec_levels_result *out) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    c->launches = 0;
    if (!out) return set_err(c, DGEC_ERR_INVALID_ARG, "out is null");
    if (n_edges < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "negative size");
    DG_TRY(check_levels(c, params));
    LvDesc d = lv_desc(n_edges, n_vertices, params);
    DG_TRY(check_batch(c, d.hb()));
    if (n_edges > 0 && (!d_src || !d_dst || !d_t)) return set_err(c, DGEC_ERR_INVALID_ARG, "null input");
    if (!d_ws || ((uintptr_t)d_ws & 255))
        return set_err(c, DGEC_ERR_INVALID_ARG, "workspace null or not 256-byte aligned");
    CU_TRY(c, cudaSetDevice(c->device));
    c->stream = (cudaStream_t)stream;
    memset(out, 0, sizeof(*out));
    const int q = params->n_levels;
    const bool dense = params->flags & DGEC_LEVELS_DENSE, condense = params->min_cluster_size != 0;
    Problem p = lv_problem(d);
    size_t need = plan_lv(nullptr, p, q, dense, condense).total;
    if (ws_bytes < need) return set_err(c, DGEC_ERR_OOM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    LvLayout L = plan_lv(d_ws, p, q, dense, condense);
    p.src = d_src;
    p.dst = d_dst;
    p.t = d_t;
    HostBatch hb = d.hb();
    DG_TRY(upload_tables(c, hb, L.eoff, L.voff, L.knn_off, L.gk, L.gM));
    p.eoff = L.eoff;
    p.voff = L.voff;
    p.knn_off = L.knn_off;
    p.gk = L.gk;
    p.gM = L.gM;
    p.egraph = L.egraph;
    tl_stream_ctas = c->stream_ctas;
    stage_start(c);
    DG_STAGE("A incidence lists", stage_csr(c, p, L.csr, L.scratch));
    DG_STAGE("B skeleton and kNN", stage_skeleton(c, p, L.csr, L.skel, L.scratch));
    DG_STAGE("L discrete levels", stage_levels(c, p, L.csr, L.skel, params->h_omega, L.lv, L.scratch));
    if (condense) {
        DG_STAGE("L rows of D", build_level_rows(c, p, L.csr, L.lv, L.scratch));
        DG_STAGE("D1 dendrogram", stage_dendro(c, p, L.csr, L.lv.rows, L.den, L.scratch));
        DG_STAGE("D2 condense and labels", stage_condense(c, p, L.lv.rows, L.den, L.cond, L.scratch));
    }
    CU_TRY(c, cudaStreamSynchronize(c->stream));
    CU_TRY(c, cudaGetLastError());
    kt_collect(c);
    stage_collect(c);
    out->sk_u = L.skel.u;
    out->sk_v = L.skel.v;
    out->sk_w = L.skel.w;
    out->n_skeleton = L.skel.n;
    out->merge_level = L.lv.mlevel;
    out->merge_parent = L.lv.mparent;
    out->n_components = L.lv.ncomp;
    out->level_labels = L.lv.dense;
    out->n_merges = L.lv.n_merges;
    out->labels = condense ? L.cond.labels : nullptr;
    out->n_clusters = condense ? L.cond.n_clusters : 0;
    return DGEC_OK;
}

}  // extern "C"
