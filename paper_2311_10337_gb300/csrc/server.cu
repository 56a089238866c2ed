// Serving runtime: lanes (host thread + CUDA stream + workspace slice) that
// continuously batch pending clustering jobs. See the serving section of
// include/dgec.h for the contract.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "stages.cuh"

namespace dgec {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    dgec_job spec;
    uint64_t ticket;
    Clock::time_point t_submit, t_done;
    int32_t n_clusters = 0;
    dgec_status status = DGEC_OK;
    bool done = false;
};

// err[0]: ids outside [0, bound); err[1]: self loops
__global__ void k_job_check(const int32_t *src, const int32_t *dst, int64_t n, int32_t bound,
                            int *err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int s = src[e], d = dst[e];
        if (s < 0 || s >= bound || d < 0 || d >= bound) atomicOr(&err[0], 1);
        else if (s == d) atomicOr(&err[1], 1);
    }
}

__global__ void k_vmark(const int32_t *src, const int32_t *dst, int64_t n, int *flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        flag[src[e]] = 1;
        flag[dst[e]] = 1;
    }
}

// dense local vertex ids (rank among the vertices the job touches), in
// place; the marks are cleared for the next job
__global__ void k_vrelabel(int32_t *src, int32_t *dst, int64_t n, const long long *vmap, int *flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int s = src[e], d = dst[e];
        src[e] = (int32_t)vmap[s];
        dst[e] = (int32_t)vmap[d];
        flag[s] = 0;
        flag[d] = 0;
    }
}

__global__ void k_copy_count(const long long *vmap, int32_t bound, long long *nv_out) {
    *nv_out = vmap[bound];
}

}  // namespace
}  // namespace dgec

using namespace dgec;

struct dgec_server;

namespace {

struct Lane {
    dgec_server *srv = nullptr;
    int index = 0;
    dgec_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    char *base = nullptr;
    size_t bytes = 0;
    // carved from the lane's slice
    int32_t *in_src = nullptr, *in_dst = nullptr;
    int64_t *in_t = nullptr;
    int *flag = nullptr;
    long long *vmap = nullptr, *scan_tmp = nullptr, *nv_dev = nullptr;
    int *err = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t cap_edges = 0;
    std::thread th;
};

}  // namespace

struct dgec_server {
    int device = 0;
    int32_t vbound = 0;
    int32_t max_batch = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<Lane *> lanes;
};

namespace {

// Largest edge count a lane can admit for a job mix (upper bounds: a job of
// n edges touches at most min(2n, bound) vertices; k up to 16).
bool mix_fits(const Lane &L, const std::vector<Job *> &mix, int32_t vbound) {
    int G = (int)mix.size();
    std::vector<int64_t> eoff(G + 1, 0);
    std::vector<int32_t> nv(G), kk(G), mm(G);
    for (int g = 0; g < G; g++) {
        const dgec_job &j = mix[g]->spec;
        eoff[g + 1] = eoff[g] + j.n_edges;
        int64_t v = 2 * j.n_edges + 1;
        nv[g] = (int32_t)(v < vbound ? v : vbound);
        kk[g] = j.k;
        mm[g] = j.min_cluster_size;
    }
    if (eoff[G] > L.cap_edges) return false;
    size_t need = 0;
    if (dgec_batch_workspace_size(G, eoff.data(), nv.data(), kk.data(), mm.data(), &need) != DGEC_OK)
        return false;
    return need <= L.ws_bytes;
}

void finish(dgec_server *s, Job *j, dgec_status st, int32_t ncl) {
    std::lock_guard<std::mutex> lk(s->mu);
    j->status = st;
    j->n_clusters = ncl;
    j->t_done = Clock::now();
    j->done = true;
    s->cv_done.notify_all();
}

void lane_loop(Lane *L) {
    dgec_server *s = L->srv;
    cudaSetDevice(s->device);
    Ctx *c = &L->ctx->c;
    c->stream = L->stream;
    for (;;) {
        std::vector<Job *> mix;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->stop && s->pending.empty()) return;
            // admission by memory, in arrival order
            while (!s->pending.empty() && (int)mix.size() < s->max_batch) {
                mix.push_back(s->pending.front());
                if (!mix_fits(*L, mix, s->vbound)) {
                    mix.pop_back();
                    break;
                }
                s->pending.pop_front();
            }
            if (mix.empty()) {
                // the head job does not fit even alone: it never will
                Job *j = s->pending.front();
                s->pending.pop_front();
                lk.unlock();
                finish(s, j, DGEC_ERR_ADMISSION, 0);
                continue;
            }
            if (!s->pending.empty()) s->cv_work.notify_one();  // let another lane take the rest
        }
        // 1. validate each job on its own arrays
        int G = (int)mix.size();
        cudaMemsetAsync(L->err, 0, sizeof(int) * 2 * G, L->stream);
        for (int g = 0; g < G; g++) {
            const dgec_job &j = mix[g]->spec;
            if (j.n_edges > 0)
                k_job_check<<<grid_for(j.n_edges, kBlock, 4096), kBlock, 0, L->stream>>>(
                    j.d_src, j.d_dst, j.n_edges, s->vbound, L->err + 2 * g);
        }
        std::vector<int> err(2 * G);
        cudaMemcpyAsync(err.data(), L->err, sizeof(int) * 2 * G, cudaMemcpyDeviceToHost, L->stream);
        if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
            for (Job *j : mix) finish(s, j, DGEC_ERR_CUDA, 0);
            continue;
        }
        std::vector<Job *> ok;
        for (int g = 0; g < G; g++) {
            if (err[2 * g]) finish(s, mix[g], DGEC_ERR_VERTEX_RANGE, 0);
            else if (err[2 * g + 1]) finish(s, mix[g], DGEC_ERR_SELF_LOOP, 0);
            else ok.push_back(mix[g]);
        }
        if (ok.empty()) continue;
        // 2. gather the jobs end to end and give each dense vertex ids
        G = (int)ok.size();
        std::vector<int64_t> eoff(G + 1, 0);
        std::vector<int32_t> kk(G), mm(G), nv(G);
        for (int g = 0; g < G; g++) {
            const dgec_job &j = ok[g]->spec;
            int64_t o = eoff[g], n = j.n_edges;
            eoff[g + 1] = o + n;
            kk[g] = j.k;
            mm[g] = j.min_cluster_size;
            if (n == 0) {
                cudaMemsetAsync(L->nv_dev + g, 0, sizeof(long long), L->stream);
                continue;
            }
            cudaMemcpyAsync(L->in_src + o, j.d_src, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, L->stream);
            cudaMemcpyAsync(L->in_dst + o, j.d_dst, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, L->stream);
            cudaMemcpyAsync(L->in_t + o, j.d_t, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, L->stream);
            k_vmark<<<grid_for(n, kBlock, 4096), kBlock, 0, L->stream>>>(L->in_src + o, L->in_dst + o, n, L->flag);
            exclusive_scan_i32(c, L->flag, L->vmap, (int64_t)s->vbound + 1, L->scan_tmp);
            k_copy_count<<<1, 1, 0, L->stream>>>(L->vmap, s->vbound, L->nv_dev + g);
            k_vrelabel<<<grid_for(n, kBlock, 4096), kBlock, 0, L->stream>>>(L->in_src + o, L->in_dst + o, n,
                                                                          L->vmap, L->flag);
        }
        std::vector<long long> nvl(G);
        cudaMemcpyAsync(nvl.data(), L->nv_dev, sizeof(long long) * G, cudaMemcpyDeviceToHost, L->stream);
        if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
            for (Job *j : ok) finish(s, j, DGEC_ERR_CUDA, 0);
            continue;
        }
        for (int g = 0; g < G; g++) nv[g] = (int32_t)(nvl[g] > 0 ? nvl[g] : 1);
        // 3. one batched pass
        dgec_batch_result br;
        dgec_status st = dgec_run_batch(L->ctx, G, eoff.data(), nv.data(), kk.data(), mm.data(), L->in_src,
                                        L->in_dst, L->in_t, L->ws, L->ws_bytes, L->stream, &br);
        if (st != DGEC_OK) {
            for (Job *j : ok) finish(s, j, st, 0);
            continue;
        }
        // 4. labels out, per-job cluster counts back
        std::vector<int32_t> ncl(G);
        for (int g = 0; g < G; g++) {
            const dgec_job &j = ok[g]->spec;
            if (j.n_edges > 0)
                cudaMemcpyAsync(j.d_labels, br.labels + eoff[g], sizeof(int32_t) * j.n_edges,
                                cudaMemcpyDeviceToDevice, L->stream);
        }
        cudaMemcpyAsync(ncl.data(), br.n_clusters, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, L->stream);
        cudaError_t e = cudaStreamSynchronize(L->stream);
        for (int g = 0; g < G; g++) finish(s, ok[g], e == cudaSuccess ? DGEC_OK : DGEC_ERR_CUDA, ncl[g]);
    }
}

}  // namespace

extern "C" {

dgec_status dgec_server_create(int device, void *d_pool, size_t pool_bytes, int32_t n_lanes,
                               int32_t vertex_bound, int32_t max_jobs_per_batch, dgec_server **out) {
    if (!out || !d_pool || ((uintptr_t)d_pool & 255) || n_lanes < 1 || vertex_bound < 2 ||
        max_jobs_per_batch < 1)
        return DGEC_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return DGEC_ERR_CUDA;
    dgec_server *s = new (std::nothrow) dgec_server();
    if (!s) return DGEC_ERR_OOM;
    s->device = device;
    s->vbound = vertex_bound;
    s->max_batch = max_jobs_per_batch;
    size_t slice = (pool_bytes / n_lanes) & ~(size_t)255;
    for (int i = 0; i < n_lanes; i++) {
        Lane *L = new Lane();
        L->srv = s;
        L->index = i;
        L->base = (char *)d_pool + slice * i;
        L->bytes = slice;
        if (dgec_create(&L->ctx, device) != DGEC_OK ||
            cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) {
            s->lanes.push_back(L);  // released with the others (no thread yet)
            dgec_server_destroy(s);
            return DGEC_ERR_CUDA;
        }
        // fixed parts: vertex renumbering scratch, error words, counts
        Arena a(L->base, slice);
        int64_t vb = vertex_bound;
        L->flag = a.take<int>(vb + 1);
        L->vmap = a.take<long long>(vb + 1);
        L->scan_tmp = a.take<long long>(scan_scratch_elems(vb + 1));
        L->err = a.take<int>(2 * (size_t)max_jobs_per_batch);
        L->nv_dev = a.take<long long>(max_jobs_per_batch);
        size_t fixed = a.off;
        if (fixed >= slice) {
            s->lanes.push_back(L);  // released with the others (no thread yet)
            dgec_server_destroy(s);
            return DGEC_ERR_OOM;
        }
        // the rest: batch input (16 B/edge) + pipeline workspace; the
        // largest edge count whose single-job workspace fits
        int64_t lo = 0, hi = int64_t(1) << 30;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) / 2;
            dgec_params pr{16, 2, 0};
            int32_t vv = (int32_t)(2 * mid + 1 < vb ? 2 * mid + 1 : vb);
            size_t w = 0;
            if (dgec_workspace_size(mid, vv, &pr, &w) == DGEC_OK &&
                fixed + 16 * (size_t)mid + 4096 + w <= slice)
                lo = mid;
            else
                hi = mid - 1;
        }
        L->cap_edges = lo;
        L->in_src = a.take<int32_t>(lo);
        L->in_dst = a.take<int32_t>(lo);
        L->in_t = a.take<int64_t>(lo);
        size_t used = (a.off + 255) & ~(size_t)255;
        L->ws = L->base + used;
        L->ws_bytes = slice > used ? slice - used : 0;
        if (cudaMemsetAsync(L->flag, 0, sizeof(int) * (vb + 1), L->stream) != cudaSuccess ||
            cudaStreamSynchronize(L->stream) != cudaSuccess) {
            s->lanes.push_back(L);  // released with the others (no thread yet)
            dgec_server_destroy(s);
            return DGEC_ERR_CUDA;
        }
        s->lanes.push_back(L);
    }
    for (Lane *L : s->lanes) L->th = std::thread(lane_loop, L);
    *out = s;
    return DGEC_OK;
}

int64_t dgec_server_lane_capacity(const dgec_server *s) {
    if (!s || s->lanes.empty()) return -1;
    return s->lanes[0]->cap_edges;
}

dgec_status dgec_submit(dgec_server *s, const dgec_job *job, uint64_t *ticket) {
    if (!s || !job || !ticket || job->n_edges < 0 || job->k < 1 || job->k > 16 ||
        job->min_cluster_size < 2)
        return DGEC_ERR_INVALID_ARG;
    if (job->n_edges > 0 && (!job->d_src || !job->d_dst || !job->d_t || !job->d_labels))
        return DGEC_ERR_INVALID_ARG;
    Job *j = new (std::nothrow) Job();
    if (!j) return DGEC_ERR_OOM;
    j->spec = *job;
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete j;
            return DGEC_ERR_INVALID_ARG;
        }
        j->ticket = s->next_ticket++;
        s->jobs[j->ticket] = j;
        s->pending.push_back(j);
    }
    s->cv_work.notify_one();
    *ticket = j->ticket;
    return DGEC_OK;
}

dgec_status dgec_wait(dgec_server *s, uint64_t ticket, int32_t timeout_ms, int32_t *n_clusters,
                      double *latency_ms) {
    if (!s) return DGEC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return DGEC_ERR_INVALID_ARG;
    Job *j = it->second;
    auto ready = [&] { return j->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return DGEC_ERR_TIMEOUT;
    dgec_status st = j->status;
    if (n_clusters) *n_clusters = j->n_clusters;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    s->jobs.erase(it);
    delete j;
    return st;
}

dgec_status dgec_server_destroy(dgec_server *s) {
    if (!s) return DGEC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // jobs never taken by a lane end with an error
        for (Job *j : s->pending) {
            j->status = DGEC_ERR_INVALID_ARG;
            j->done = true;
        }
        s->pending.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (Lane *L : s->lanes) {
        if (L->th.joinable()) L->th.join();
        if (L->stream) cudaStreamDestroy(L->stream);
        if (L->ctx) dgec_destroy(L->ctx);
        delete L;
    }
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return DGEC_OK;
}

}  // extern "C"
