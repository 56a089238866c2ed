// Stage A: incidence lists (Alg. 3, first line: "Generate adjacency list
// representation") with every vertex's in-list and out-list sorted by time
// (Alg. 2: "Sort E_i by time"; ties by edge id).
//
// First a device-wide radix sort of the 64-bit keys ((t - t_min) << idbits
// | id) ranks all edges in (t, id) order. The keys are laid out in id order
// and the LSD sort is stable, so only the time bits need passes: equal
// times keep id order. That rank r is the internal node
// id of every later stage, and per-vertex lists sorted by (t, id) are just
// lists sorted by r. Ranks are scattered into their vertex's segment through
// per-vertex cursors (warp-aggregated atomics absorb hub vertices), then
// each segment is sorted by the bin its length falls in:
//   2..32 elements      one warp, bitonic network over shuffles;
//   33..256, 257..2048  one CTA, bitonic network in shared memory;
//   > 2048 (hubs)       all hub segments together through the device-wide
//                       radix sort, keyed (segment, r).
#include "stages.cuh"

namespace dgec {

constexpr unsigned long long kPad = 0xFFFFFFFFFFFFFFFFull;

// flags: [0] bad vertex count, [1] self loop count, [2] t min, [3] t max
// graph of every edge (binary search over the batch's edge offsets)
__global__ void k_egraph(const int64_t *eoff, int G, int64_t E, int32_t *egraph) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;  // last g with eoff[g] <= e
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (eoff[mid] <= e) lo = mid;
            else hi = mid;
        }
        egraph[e] = lo;
    }
}

// Validates ids against each edge's own graph and counts degrees under
// global vertex ids (local id + the graph's vertex offset).
__global__ void k_count(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E,
                        const int32_t *egraph, const int64_t *voff, int *deg_out, int *deg_in,
                        long long *flags) {
    __shared__ long long smin[kBlock / 32], smax[kBlock / 32];
    long long tmin = LLONG_MAX, tmax = LLONG_MIN;
    int bad = 0, loops = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-aligned grid-stride loop so warp_agg_inc sees whole warps
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = stride >> 5;
    for (int64_t wb = warp_global * 32; wb < E; wb += nwarps * 32) {
        int64_t e = wb + lane_id();
        bool ok = e < E;
        int s = ok ? src[e] : 0, d = ok ? dst[e] : 0;
        int64_t vo = 0, nv = 0;
        if (ok) {
            int g = egraph[e];
            vo = voff[g];
            nv = voff[g + 1] - vo;
        }
        bool vs = ok && s >= 0 && s < nv && d >= 0 && d < nv;
        if (ok && !vs) bad++;
        if (vs && s == d) loops++;
        if (ok) {
            long long x = t[e];
            tmin = x < tmin ? x : tmin;
            tmax = x > tmax ? x : tmax;
        }
        unsigned act = __ballot_sync(0xffffffffu, vs);
        if (vs) {
            warp_agg_inc(deg_out, (int)(s + vo), act);
            warp_agg_inc(deg_in, (int)(d + vo), act);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long a = __shfl_xor_sync(0xffffffffu, tmin, o);
        long long b = __shfl_xor_sync(0xffffffffu, tmax, o);
        tmin = a < tmin ? a : tmin;
        tmax = b > tmax ? b : tmax;
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        loops += __shfl_xor_sync(0xffffffffu, loops, o);
    }
    if (lane_id() == 0) {
        smin[threadIdx.x >> 5] = tmin;
        smax[threadIdx.x >> 5] = tmax;
        if (bad) atomicAdd((unsigned long long *)&flags[0], (unsigned long long)bad);
        if (loops) atomicAdd((unsigned long long *)&flags[1], (unsigned long long)loops);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            tmin = smin[w] < tmin ? smin[w] : tmin;
            tmax = smax[w] > tmax ? smax[w] : tmax;
        }
        tmin = smin[0] < tmin ? smin[0] : tmin;
        tmax = smax[0] > tmax ? smax[0] : tmax;
        atomicMin(&flags[2], tmin);
        atomicMax(&flags[3], tmax);
    }
}

__global__ void k_init_flags(long long *flags) {
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = LLONG_MAX;
    flags[3] = LLONG_MIN;
}

__global__ void k_set_i64(long long *p, long long v) { *p = v; }

// rank r = position of edge (t, id) in the global order; time-ordered
// copies of the inputs for the later stages
__global__ void k_rank_init(const unsigned long long *ks, int64_t E, long long tmin, int idbits,
                            const int32_t *src, const int32_t *dst, const int32_t *egraph,
                            const int64_t *voff, int32_t *orig_of, int32_t *rank_of, int32_t *isrc,
                            int32_t *idst, int64_t *it) {
    const unsigned long long idmask = (1ull << idbits) - 1ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = ks[r];
        int32_t e = (int32_t)(k & idmask);
        orig_of[r] = e;
        rank_of[e] = (int32_t)r;
        it[r] = (int64_t)(k >> idbits) + tmin;
        int32_t vo = (int32_t)voff[egraph[e]];
        isrc[r] = src[e] + vo;
        idst[r] = dst[e] + vo;
    }
}

__global__ void k_pack_keys(const int64_t *t, int64_t E, long long tmin, int idbits,
                            unsigned long long *k) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        k[e] = ((unsigned long long)(t[e] - tmin) << idbits) | (unsigned long long)e;
}

__global__ void k_scatter(const int32_t *isrc, const int32_t *idst, int64_t E,
                          const int64_t *out_off, const int64_t *in_off, int *cur_out, int *cur_in,
                          unsigned long long *okey, unsigned long long *ikey) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = stride >> 5;
    for (int64_t wb = warp_global * 32; wb < E; wb += nwarps * 32) {
        int64_t r = wb + lane_id();
        bool ok = r < E;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            int s = isrc[r], d = idst[r];
            int ro = warp_agg_inc(cur_out, s, act);
            int ri = warp_agg_inc(cur_in, d, act);
            okey[out_off[s] + ro] = (unsigned long long)r;
            ikey[in_off[d] + ri] = (unsigned long long)r;
        }
    }
}

// bins: 0 warp (2..32), 1 CTA-256, 2 CTA-2048, 3 hub (> 2048)
__global__ void k_classify(const int64_t *off, int64_t V, int *bin_cnt, int *bin_list,
                           int64_t list_stride) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t wb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; wb < V;
         wb += stride) {
        int64_t v = wb + lane_id();
        int b = -1;
        if (v < V) {
            int64_t d = off[v + 1] - off[v];
            b = d <= 1 ? -1 : d <= 32 ? 0 : d <= 256 ? 1 : d <= 2048 ? 2 : 3;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            unsigned m = __ballot_sync(0xffffffffu, b == q);
            if (m == 0) continue;
            int leader = __ffs(m) - 1;
            int base = 0;
            if ((int)lane_id() == leader) base = atomicAdd(&bin_cnt[q], __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (b == q) bin_list[q * list_stride + base + __popc(m & ((1u << lane_id()) - 1u))] = (int)v;
        }
    }
}

// One warp per segment of 2..32 keys: bitonic sort across lanes.
__global__ void k_sort_warp(unsigned long long *keys, const int64_t *off, const int *list, int n) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    int v = list[w];
    int64_t b = off[v];
    int d = (int)(off[v + 1] - b);
    unsigned l = lane_id();
    unsigned long long x = (int)l < d ? keys[b + l] : kPad;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            unsigned long long y = __shfl_xor_sync(0xffffffffu, x, stride);
            bool up = (l & size) == 0;        // this lane's run sorts ascending
            bool low = (l & stride) == 0;     // this lane holds the lower slot
            bool take_min = (up == low);
            x = take_min ? (x < y ? x : y) : (x > y ? x : y);
        }
    }
    if ((int)l < d) keys[b + l] = x;
}

// One CTA per segment of up to CAP keys: bitonic sort in shared memory.
template <int CAP>
__global__ void k_sort_block(unsigned long long *keys, const int64_t *off, const int *list) {
    __shared__ unsigned long long s[CAP];
    int v = list[blockIdx.x];
    int64_t b = off[v];
    int d = (int)(off[v + 1] - b);
    int N = 1;
    while (N < d) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = i < d ? keys[b + i] : kPad;
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                int lo = 2 * stride * (i / stride) + (i % stride);
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                unsigned long long a = s[lo], c = s[hi];
                if ((a > c) == up) {
                    s[lo] = c;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x) keys[b + i] = s[i];
}

__global__ void k_hub_sizes(const int64_t *off, const int *list, int n, long long *sz) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sz[i] = off[list[i] + 1] - off[list[i]];
    if (i == n) sz[i] = 0;
}

// Copy hub segments into one array: key = list key, value = hub index.
__global__ void k_hub_gather(const unsigned long long *keys, const int64_t *off, const int *list,
                             int nh, const long long *hoff, unsigned long long *hk,
                             unsigned long long *hv) {
    for (int h = blockIdx.y; h < nh; h += gridDim.y) {
        int v = list[h];
        int64_t b = off[v], d = off[v + 1] - b, o = hoff[h];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d;
             i += (int64_t)gridDim.x * blockDim.x) {
            hk[o + i] = keys[b + i];
            hv[o + i] = (unsigned long long)h;
        }
    }
}

// After sorting by (hub, key): element j goes back to its hub's segment.
__global__ void k_hub_scatter(const unsigned long long *hub_of, const unsigned long long *key_of,
                              int64_t n, const int64_t *off, const int *list,
                              const long long *hoff, unsigned long long *keys) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        int h = (int)hub_of[j];
        keys[off[list[h]] + (j - hoff[h])] = key_of[j];
    }
}

__global__ void k_unpack(const unsigned long long *keys, int64_t E, const int32_t *orig_of,
                         const int64_t *it, int64_t *t_out, int32_t *id_out, int32_t *r_out,
                         int32_t *slot_of, int32_t *pos_of) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = (int32_t)keys[x];
        const int32_t e = orig_of[r];
        r_out[x] = r;
        id_out[x] = e;
        t_out[x] = it[r];
        if (slot_of) slot_of[r] = (int32_t)x;
        pos_of[e] = (int32_t)x;  // the edge's place in this list array
    }
}

void plan_csr(Arena &ws, const Problem &p, Csr &o) {
    o.out_off = ws.take<int64_t>(p.V + 1);
    o.in_off = ws.take<int64_t>(p.V + 1);
    o.out_t = ws.take<int64_t>(p.E);
    o.in_t = ws.take<int64_t>(p.E);
    o.out_id = ws.take<int32_t>(p.E);
    o.in_id = ws.take<int32_t>(p.E);
    o.out_r = ws.take<int32_t>(p.E);
    o.in_r = ws.take<int32_t>(p.E);
    o.orig_of = ws.take<int32_t>(p.E);
    o.rank_of = ws.take<int32_t>(p.E);
    o.isrc = ws.take<int32_t>(p.E);
    o.idst = ws.take<int32_t>(p.E);
    o.it = ws.take<int64_t>(p.E);
    o.slot_out = ws.take<int32_t>(p.E);
    o.pos_out = ws.take<int32_t>(p.E);
    o.pos_in = ws.take<int32_t>(p.E);
}

void carve_segsort(Arena &a, int64_t V, int64_t n, SegSort &s) {
    s.bin_cnt = a.take<int>(8);
    s.bin_list = a.take<int>(4 * (V + 1));
    s.scan_tmp = a.take<long long>(scan_scratch_elems(n / 2048 + 8));
    s.hoff = a.take<long long>(n / 2048 + 8);
    s.hsz = a.take<long long>(n / 2048 + 8);
    s.hk = a.take<unsigned long long>(n);
    s.hv = a.take<unsigned long long>(n);
    s.hk2 = a.take<unsigned long long>(n);
    s.hv2 = a.take<unsigned long long>(n);
    s.radix = a.take<char>(radix_scratch_bytes(n));
}

// scratch layout
struct CsrScratch {
    int *deg_out, *deg_in;
    long long *flags, *scan_tmp;
    unsigned long long *okey, *ikey;
    SegSort seg;
    void *radix;
};
static CsrScratch carve_csr(Arena &a, const Problem &p) {
    CsrScratch s;
    int64_t V = p.V, E = p.E;
    s.deg_out = a.take<int>(V + 1);
    s.deg_in = a.take<int>(V + 1);
    s.flags = a.take<long long>(8);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(V + 1));
    s.okey = a.take<unsigned long long>(E);
    s.ikey = a.take<unsigned long long>(E);
    carve_segsort(a, V, E, s.seg);
    s.radix = a.take<char>(radix_scratch_bytes(E));
    return s;
}

size_t csr_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_csr(a, p);
    return a.off;
}

dgec_status sort_segments(Ctx *c, int64_t V, unsigned long long *keys, const int64_t *off, SegSort &s,
                          int key_bits) {
    cudaStream_t st = c->stream;
    CU_TRY(c, cudaMemsetAsync(s.bin_cnt, 0, 8 * sizeof(int), st));
    TK(c, "k_classify", k_classify<<<grid_for(V, kBlock, 8192), kBlock, 0, st>>>(off, V, s.bin_cnt, s.bin_list, V + 1));
    int64_t h[4];
    CU_TRY(c, cudaMemcpyAsync(c->h_pinned, s.bin_cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CU_TRY(c, cudaStreamSynchronize(st));
    {
        int tmp[4];
        memcpy(tmp, c->h_pinned, sizeof(tmp));
        for (int q = 0; q < 4; q++) h[q] = tmp[q];
    }
    if (h[0]) {
        TK(c, "k_sort_warp", k_sort_warp<<<grid_for(h[0] * 32), kBlock, 0, st>>>(keys, off, s.bin_list, (int)h[0]));
    }
    if (h[1]) {
        TK(c, "k_sort_block<256>", k_sort_block<256><<<(unsigned)h[1], 128, 0, st>>>(keys, off, s.bin_list + (V + 1)));
    }
    if (h[2]) {
        TK(c, "k_sort_block<2048>", k_sort_block<2048><<<(unsigned)h[2], 1024, 0, st>>>(keys, off, s.bin_list + 2 * (V + 1)));
    }
    if (h[3]) {
        const int *hl = s.bin_list + 3 * (V + 1);
        int nh = (int)h[3];
        TK(c, "k_hub_sizes", k_hub_sizes<<<grid_for(nh + 1), kBlock, 0, st>>>(off, hl, nh, s.hsz));
        DG_TRY(exclusive_scan_i64(c, s.hsz, s.hoff, nh + 1, s.scan_tmp));
        int64_t tot;
        DG_TRY(read_counters(c, (const int64_t *)(s.hoff + nh), 1, &tot));
        long long *hstart = s.hoff;
        dim3 g((unsigned)grid_for(2048 * 64, kBlock, 64), (unsigned)(nh < 65535 ? nh : 65535));
        TK(c, "k_hub_gather", k_hub_gather<<<g, kBlock, 0, st>>>(keys, off, hl, nh, hstart, s.hk, s.hv));
        bool in_b;
        RadixBuffers rb{s.hk, s.hk2, s.hv, s.hv2};
        DG_TRY(radix_sort(c, rb, tot, 0, key_bits, s.radix, &in_b));
        unsigned long long *k1 = in_b ? s.hk2 : s.hk, *v1 = in_b ? s.hv2 : s.hv;
        unsigned long long *k1o = in_b ? s.hk : s.hk2, *v1o = in_b ? s.hv : s.hv2;
        // second pass: stable by hub index (payload = key)
        RadixBuffers rb2{v1, v1o, k1, k1o};
        int hb = bits_for((uint64_t)(nh - 1));
        if (hb == 0) hb = 1;
        DG_TRY(radix_sort(c, rb2, tot, 0, hb, s.radix, &in_b));
        unsigned long long *hub_of = in_b ? v1o : v1, *key_of = in_b ? k1o : k1;
        TK(c, "k_hub_scatter", k_hub_scatter<<<grid_for(tot, kBlock, 65536), kBlock, 0, st>>>(hub_of, key_of, tot, off, hl, hstart,
                                                                       keys));
    }
    return DGEC_OK;
}

dgec_status stage_csr(Ctx *c, Problem &p, Csr &o, void *scratch) {
    cudaStream_t st = c->stream;
    Arena a(scratch, SIZE_MAX);
    CsrScratch s = carve_csr(a, p);
    int64_t V = p.V, E = p.E;
    CU_TRY(c, cudaMemsetAsync(s.deg_out, 0, sizeof(int) * (V + 1), st));
    CU_TRY(c, cudaMemsetAsync(s.deg_in, 0, sizeof(int) * (V + 1), st));
    TK(c, "k_init_flags", k_init_flags<<<1, 1, 0, st>>>(s.flags));
    if (E > 0) {
        if (p.G == 1) CU_TRY(c, cudaMemsetAsync(p.egraph, 0, sizeof(int32_t) * E, st));
        else TK(c, "k_egraph", k_egraph<<<grid_for(E, kBlock, 65536), kBlock, 0, st>>>(p.eoff, p.G, E, p.egraph));
        TK(c, "k_count", k_count<<<grid_for(E, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                             p.src, p.dst, p.t, E, p.egraph, p.voff, s.deg_out, s.deg_in, s.flags));
    }
    int64_t f[4];
    DG_TRY(read_counters(c, (const int64_t *)s.flags, 4, f));
    if (f[0]) return set_err(c, DGEC_ERR_VERTEX_RANGE, "%lld edges have a vertex id outside their graph's range",
                             (long long)f[0]);
    if (f[1]) return set_err(c, DGEC_ERR_SELF_LOOP, "%lld self loops (i, i, t)", (long long)f[1]);
    p.tmin = E > 0 ? f[2] : 0;
    uint64_t span = E > 0 ? (uint64_t)(f[3] - f[2]) : 0;
    p.idbits = bits_for((uint64_t)(E > 1 ? E - 1 : 1));
    p.tbits = bits_for(span);
    if (p.idbits + p.tbits > 64)
        return set_err(c, DGEC_ERR_TOO_LARGE, "time span %llu needs %d bits + %d id bits > 64",
                       (unsigned long long)span, p.tbits, p.idbits);
    // offsets
    if (V > 0) {
        DG_TRY(exclusive_scan_i32(c, s.deg_out, (long long *)o.out_off, V, s.scan_tmp));
        DG_TRY(exclusive_scan_i32(c, s.deg_in, (long long *)o.in_off, V, s.scan_tmp));
    }
    TK(c, "k_set_i64", k_set_i64<<<1, 1, 0, st>>>((long long *)o.out_off + V, E));
    TK(c, "k_set_i64", k_set_i64<<<1, 1, 0, st>>>((long long *)o.in_off + V, E));
    if (E == 0) return DGEC_OK;
    // global (t, id) order: internal ids
    const int gEE = grid_for(E, kBlock, 65536);
    TK(c, "k_pack_keys", k_pack_keys<<<gEE, kBlock, 0, st>>>(p.t, E, p.tmin, p.idbits, s.okey));
    {
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.okey, s.ikey, nullptr, nullptr}, E, p.idbits, p.idbits + p.tbits,
                          s.radix, &in_b));
        TK(c, "k_rank_init", k_rank_init<<<gEE, kBlock, 0, st>>>(in_b ? s.ikey : s.okey, E, p.tmin, p.idbits,
                                                                p.src, p.dst, p.egraph, p.voff, o.orig_of, o.rank_of,
                                                                o.isrc, o.idst, o.it));
    }
    // scatter ranks into their segments (cursors reuse the degree arrays)
    CU_TRY(c, cudaMemsetAsync(s.deg_out, 0, sizeof(int) * (V + 1), st));
    CU_TRY(c, cudaMemsetAsync(s.deg_in, 0, sizeof(int) * (V + 1), st));
    TK(c, "k_scatter", k_scatter<<<grid_for(E, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                           o.isrc, o.idst, E, o.out_off, o.in_off, s.deg_out, s.deg_in, s.okey, s.ikey));
    DG_TRY(sort_segments(c, V, s.okey, o.out_off, s.seg, p.idbits));
    DG_TRY(sort_segments(c, V, s.ikey, o.in_off, s.seg, p.idbits));
    TK(c, "k_unpack", k_unpack<<<gEE, kBlock, 0, st>>>(s.okey, E, o.orig_of, o.it, o.out_t, o.out_id,
                                                       o.out_r, o.slot_out, o.pos_out));
    TK(c, "k_unpack", k_unpack<<<gEE, kBlock, 0, st>>>(s.ikey, E, o.orig_of, o.it, o.in_t, o.in_id,
                                                       o.in_r, nullptr, o.pos_in));
    return DGEC_OK;
}

}  // namespace dgec
