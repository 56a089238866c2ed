// dgec_msf_static: the Borůvka minimum-spanning-forest stage with its
// working memory in a fixed, file-scope device array instead of a
// caller-supplied workspace.
//
// Who needs this: callers that may not allocate device memory at the point
// where they want a forest -- code that runs inside a framework which owns
// every device allocation (a plugin or an inference server with a
// pre-reserved pool), real-time loops that forbid allocation after start-up,
// and hosts that cannot reach cudaMalloc at all from the calling thread. The
// array below is reserved once, when the library is loaded onto a device,
// and stays reserved on every device that loads the library until the
// process exits.
//
// Limits: at most kStaticMaxNodes nodes and kStaticMaxEdges edges per call;
// larger inputs are rejected with DGEC_ERR_TOO_LARGE.
//
// Sharing: every call uses the same array and leaves its contents behind;
// each call re-initialises the parts that must start from a known value
// (labels, best-edge slots, counters). Two calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race on
// the array and give wrong results; serialise them.
#include <mutex>

#include "stages.cuh"

namespace dgec {

// Borůvka kernels defined in msf.cu.
__global__ void k_filter_bid(const int32_t *u, const int32_t *v, const int64_t *w, int64_t n,
                             const int32_t *comp, int32_t *u2, int32_t *v2, int64_t *w2,
                             unsigned long long *cnt, unsigned long long *bw);
__global__ void k_bid_uv(const int32_t *u, const int32_t *v, const int64_t *w, int64_t n,
                         const int32_t *comp, const unsigned long long *bw, unsigned long long *buv);
__global__ void k_hook(int64_t E, const int32_t *comp, const unsigned long long *bw,
                       const unsigned long long *buv, int32_t *par, int32_t *mu, int32_t *mv,
                       int64_t *mw, unsigned long long *n_out);
__global__ void k_jump(int64_t E, const int32_t *comp, int32_t *par);
__global__ void k_relabel(int64_t E, int32_t *comp, const int32_t *par, unsigned long long *bw,
                          unsigned long long *buv);
__global__ void k_reset_best(int64_t E, unsigned long long *bw, unsigned long long *buv);
__global__ void k_iota(int64_t E, int32_t *comp);

constexpr int64_t kStaticMaxNodes = int64_t(1) << 18;  // 262,144 nodes
constexpr int64_t kStaticMaxEdges = int64_t(1) << 19;  // 524,288 edges

// Byte layout of the static array (each part 256-byte aligned).
constexpr size_t kAl = 256;
constexpr size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }
constexpr size_t kOffComp = 0;
constexpr size_t kOffPar = kOffComp + al(kStaticMaxNodes * 4);
constexpr size_t kOffBw = kOffPar + al(kStaticMaxNodes * 4);
constexpr size_t kOffBuv = kOffBw + al(kStaticMaxNodes * 8);
constexpr size_t kOffUa = kOffBuv + al(kStaticMaxNodes * 8);
constexpr size_t kOffVa = kOffUa + al(kStaticMaxEdges * 4);
constexpr size_t kOffWa = kOffVa + al(kStaticMaxEdges * 4);
constexpr size_t kOffUb = kOffWa + al(kStaticMaxEdges * 8);
constexpr size_t kOffVb = kOffUb + al(kStaticMaxEdges * 4);
constexpr size_t kOffWb = kOffVb + al(kStaticMaxEdges * 4);
constexpr size_t kOffCnt = kOffWb + al(kStaticMaxEdges * 8);
constexpr size_t kStaticBytes = kOffCnt + al(4 * 8);  // about 22 MB

static __device__ __align__(256) unsigned char g_msf_scratch[kStaticBytes];

// Checks the caller's edge list: counter[0] += edges with an id out of
// range, with u >= v, or with a negative weight (weights are compared as
// unsigned in the bids, so w < 0 would sort after every valid weight).
__global__ void k_static_check(const int32_t *u, const int32_t *v, const int64_t *w, int64_t n,
                               int64_t n_nodes, unsigned long long *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int a = u[x], b = v[x];
        if (a < 0 || b >= n_nodes || a >= b || w[x] < 0) atomicAdd(bad, 1ull);
    }
}

// Device address of the static array, looked up once per device (host code
// only sees a host-side stand-in for the symbol).
static std::mutex g_addr_mu;
static void *g_addr[64];

static dgec_status static_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= 64) return DGEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_msf_scratch) != cudaSuccess || !p) return DGEC_ERR_CUDA;
        g_addr[device] = p;
    }
    *out = (unsigned char *)g_addr[device];
    return DGEC_OK;
}

static dgec_status read_u64(cudaStream_t st, const unsigned long long *d, unsigned long long *h) {
    if (cudaMemcpyAsync(h, d, sizeof(*h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DGEC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DGEC_ERR_CUDA;
    return DGEC_OK;
}

}  // namespace dgec

using namespace dgec;

extern "C" dgec_status dgec_msf_static(const int32_t *d_u, const int32_t *d_v, const int64_t *d_w,
                                       int64_t n_edges, int64_t n_nodes, int32_t *d_mst_u,
                                       int32_t *d_mst_v, int64_t *d_mst_w, int64_t *h_n_mst,
                                       void *cuda_stream) {
    if (n_edges < 0 || n_nodes < 0 || !h_n_mst) return DGEC_ERR_INVALID_ARG;
    if (n_nodes > kStaticMaxNodes || n_edges > kStaticMaxEdges) return DGEC_ERR_TOO_LARGE;
    if (n_edges > 0 && (!d_u || !d_v || !d_w)) return DGEC_ERR_INVALID_ARG;
    if (n_nodes > 1 && (!d_mst_u || !d_mst_v || !d_mst_w)) return DGEC_ERR_INVALID_ARG;
    *h_n_mst = 0;
    if (n_nodes == 0 || n_edges == 0) return DGEC_OK;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return DGEC_ERR_CUDA;
    unsigned char *base = nullptr;
    dgec_status s = static_scratch(device, &base);
    if (s != DGEC_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int32_t *comp = (int32_t *)(base + kOffComp), *par = (int32_t *)(base + kOffPar);
    unsigned long long *bw = (unsigned long long *)(base + kOffBw);
    unsigned long long *buv = (unsigned long long *)(base + kOffBuv);
    int32_t *ua = (int32_t *)(base + kOffUa), *va = (int32_t *)(base + kOffVa);
    int64_t *wa = (int64_t *)(base + kOffWa);
    int32_t *ub = (int32_t *)(base + kOffUb), *vb = (int32_t *)(base + kOffVb);
    int64_t *wb = (int64_t *)(base + kOffWb);
    unsigned long long *cnt = (unsigned long long *)(base + kOffCnt);  // [0] live/bad, [1] out
    // clear what must start from a known value: counters, labels, best slots
    if (cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) return DGEC_ERR_CUDA;
    k_static_check<<<grid_for(n_edges), kBlock, 0, st>>>(d_u, d_v, d_w, n_edges, n_nodes, cnt);
    if (cudaGetLastError() != cudaSuccess) return DGEC_ERR_CUDA;
    unsigned long long bad = 0;
    if ((s = read_u64(st, cnt, &bad)) != DGEC_OK) return s;
    if (bad) return DGEC_ERR_INVALID_ARG;
    const int gN = grid_for(n_nodes);
    k_iota<<<gN, kBlock, 0, st>>>(n_nodes, comp);
    k_reset_best<<<gN, kBlock, 0, st>>>(n_nodes, bw, buv);
    if (cudaGetLastError() != cudaSuccess) return DGEC_ERR_CUDA;
    const int32_t *cu = d_u, *cv = d_v;
    const int64_t *cw = d_w;
    int32_t *nu = ua, *nv = va;
    int64_t *nw = wa;
    int64_t n = n_edges;
    for (int round = 0;; round++) {
        if (round >= 64) return DGEC_ERR_TIMEOUT;
        if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st) != cudaSuccess) return DGEC_ERR_CUDA;
        k_filter_bid<<<grid_for(n), kBlock, 0, st>>>(cu, cv, cw, n, comp, nu, nv, nw, cnt, bw);
        if (cudaGetLastError() != cudaSuccess) return DGEC_ERR_CUDA;
        unsigned long long live = 0;
        if ((s = read_u64(st, cnt, &live)) != DGEC_OK) return s;
        if (live == 0) break;
        k_bid_uv<<<grid_for((int64_t)live), kBlock, 0, st>>>(nu, nv, nw, (int64_t)live, comp, bw, buv);
        k_hook<<<gN, kBlock, 0, st>>>(n_nodes, comp, bw, buv, par, d_mst_u, d_mst_v, d_mst_w, cnt + 1);
        k_jump<<<gN, kBlock, 0, st>>>(n_nodes, comp, par);
        k_relabel<<<gN, kBlock, 0, st>>>(n_nodes, comp, par, bw, buv);
        k_reset_best<<<gN, kBlock, 0, st>>>(n_nodes, bw, buv);
        if (cudaGetLastError() != cudaSuccess) return DGEC_ERR_CUDA;
        cu = nu;
        cv = nv;
        cw = nw;
        n = (int64_t)live;
        nu = (nu == ua) ? ub : ua;
        nv = (nv == va) ? vb : va;
        nw = (nw == wa) ? wb : wa;
    }
    unsigned long long m = 0;
    if ((s = read_u64(st, cnt + 1, &m)) != DGEC_OK) return s;
    *h_n_mst = (int64_t)m;
    return DGEC_OK;
}
