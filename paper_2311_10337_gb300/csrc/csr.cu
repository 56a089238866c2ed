// Stage A: incidence lists (the adjacency lists Alg. 3 starts from) with
// every vertex's in-list and out-list sorted by time as Alg. 2 needs them
// (ties by edge id), and the two merge ranks Alg. 2's sweep depends on.
//
// First a device-wide radix sort of the 64-bit keys ((t - t_min) << idbits
// | id) ranks all edges in (t, id) order. The keys are laid out in id order
// and the LSD sort is stable, so only the time bits need passes: equal
// times keep id order. That rank r is the internal node id of every later
// stage. (When the time span and the ids do not fit one 64-bit key, the
// time alone is the key and the id rides along as the sort's value: the
// same order, one more word per pass.)
//
// Then every edge contributes two incidence items: an in-item at its head
// and an out-item at its tail. Laid out in the order (t, in-before-out, r)
// -- the order Alg. 2 sweeps a vertex's merged list in, in-edges first at
// equal times -- and sorted stably over the vertex bits alone, the items
// form every vertex's merged list. From it, by positions alone and with no
// search:
//   - the out-list (in-list) of v is the sequence of out-items (in-items)
//     of v's segment, already in (t, id) order;
//   - b of an out-item q = the in-items before it in the segment
//     = #{in-edges p of v : t_p <= t_q};
//   - a of an in-item p = the out-items before it in the segment
//     = #{out-edges q of v : t_q < t_p}.
// No atomics and no per-segment sorts, so hub vertices cost nothing extra.
//
// The segment sort below (bins by length: one warp for 2..32 keys, one CTA
// for 33..2048, hubs through the radix sort keyed (segment, key)) serves the
// hypergraph membership lists, whose members arrive unordered.
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
        if (deg_out) {  // degrees only when the caller wants them
            unsigned act = __ballot_sync(0xffffffffu, vs);
            if (vs) {
                warp_agg_inc(deg_out, (int)(s + vo), act);
                warp_agg_inc(deg_in, (int)(d + vo), act);
            }
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

// (t, original id) of an internal id r in one 16-byte record, for the
// merged-list unpack's random reads by r (one sector instead of two)
struct TE {
    int64_t t;
    int32_t e, pad;
};

// rank r = position of edge (t, id) in the global order; time-ordered
// copies of the inputs for the later stages. The sort carried each edge's
// (src, dst) pair, in global vertex ids, as its value.
__global__ void k_rank_init(const unsigned long long *ks, const unsigned long long *vs, int64_t E,
                            long long tmin, int idbits, int32_t *orig_of, int32_t *rank_of, int32_t *isrc,
                            int32_t *idst, int64_t *it, TE *te) {
    const unsigned long long idmask = (1ull << idbits) - 1ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ks[r], sd = vs[r];
        const int32_t e = (int32_t)(k & idmask);
        const int64_t tt = (int64_t)(k >> idbits) + tmin;
        orig_of[r] = e;
        rank_of[e] = (int32_t)r;
        it[r] = tt;
        if (te) te[r] = TE{tt, e, 0};  // only when the merged sort cannot carry (t, id)
        isrc[r] = (int32_t)(sd & 0xffffffffull);
        idst[r] = (int32_t)(sd >> 32);
    }
}

// the same from a (t - tmin) key sorted with the edge id as its value
__global__ void k_rank_init_kv(const unsigned long long *ks, const unsigned long long *vs, int64_t E,
                               long long tmin, const int32_t *src, const int32_t *dst,
                               const int32_t *egraph, const int64_t *voff, int G, int32_t *orig_of,
                               int32_t *rank_of, int32_t *isrc, int32_t *idst, int64_t *it, TE *te) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = (int32_t)vs[r];
        orig_of[r] = e;
        rank_of[e] = (int32_t)r;
        it[r] = (int64_t)(long long)(ks[r] + (unsigned long long)tmin);
        if (te) te[r] = TE{it[r], e, 0};
        int32_t vo = G > 1 ? (int32_t)voff[egraph[e]] : 0;
        isrc[r] = src[e] + vo;
        idst[r] = dst[e] + vo;
    }
}

__global__ void k_pack_t(const int64_t *t, int64_t E, long long tmin, unsigned long long *k,
                         unsigned long long *v) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        k[e] = (unsigned long long)t[e] - (unsigned long long)tmin;
        v[e] = (unsigned long long)e;
    }
}

// Time groups of the (t, id) order: flag[r] = 1 where a new time starts.
__global__ void k_thead(const int64_t *it, int64_t E, int *flag) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= E;
         r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = r < E && (r == 0 || it[r] != it[r - 1]);
}
// gstart[g] = first r of time group g; gstart[#groups] = E
__global__ void k_tgstart(const int *flag, const long long *gpos, int64_t E, int32_t *gstart) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= E;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r == E) gstart[gpos[E]] = (int32_t)E;
        else if (flag[r]) gstart[gpos[r]] = (int32_t)r;
    }
}
// Incidence items in the order (t, in-before-out, r): time group [gs, ge)
// puts its in-items at 2 gs + (r - gs) and its out-items after them.
// key = (vertex << cb) | (2 r + dir), dir 0 = in-item (at dst), 1 = out-item.
// With val (time spans below 2^32): each item also carries (original id,
// t - tmin) as its sort value, so the unpack reads nothing at random.
__global__ void k_mkeys(const int32_t *isrc, const int32_t *idst, const int *flag, const long long *gpos,
                        const int32_t *gstart, int64_t E, int cb, unsigned long long *key,
                        const int32_t *orig_of, const int64_t *it, long long tmin, unsigned long long *val) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const long long g = gpos[r] + flag[r] - 1;
        const int64_t gs = gstart[g], ge = gstart[g + 1];
        const unsigned long long code = 2ull * (unsigned long long)r;
        key[r + gs] = ((unsigned long long)(unsigned)idst[r] << cb) | code;
        key[r + ge] = ((unsigned long long)(unsigned)isrc[r] << cb) | (code | 1ull);
        if (val) {
            const unsigned long long te = ((unsigned long long)(unsigned)orig_of[r] << 32) |
                                          (unsigned long long)(it[r] - tmin);
            val[r + gs] = te;
            val[r + ge] = te;
        }
    }
}
// out_off[v] = out-items before v's segment; in_off[v] = in-items before it
__global__ void k_moff_split(const int64_t *moff, const int32_t *oidx, int64_t V, int64_t *out_off,
                             int64_t *in_off) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = moff[v];
        const int64_t o = oidx[m];
        out_off[v] = o;
        in_off[v] = m - o;
    }
}
// Every item of the merged lists goes to its slot in the out- or in-list
// arrays; its rank in the other list is its position difference.
__global__ void k_munpack(const unsigned long long *key, const unsigned long long *val, long long tmin,
                          int64_t n2, int cb, const int64_t *moff,
                          const int32_t *oidx, const int64_t *out_off, const TE *te, int64_t *out_t,
                          int32_t *out_id, int32_t *out_r, int4 *outrk, int32_t *pos_out, int64_t *in_t,
                          int32_t *in_id, int32_t *in_r, int32_t *pos_in, unsigned char *in_head,
                          int2 *inrk, int2 *in_va, int2 *out_vb, unsigned long long *out_key,
                          unsigned long long *in_key) {
    const unsigned long long cmask = (1ull << cb) - 1ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n2;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[x];
        const int64_t v = (int64_t)(k >> cb);
        const unsigned long long code = k & cmask;
        const int32_t r = (int32_t)(code >> 1);
        const int64_t ob = oidx[x];              // out-items before x
        const int64_t seg = x - moff[v];         // position in v's merged list
        const int64_t obv = ob - out_off[v];     // out-items before x within v's list
        int32_t e;
        int64_t tt;
        unsigned long long pk = 0;  // (t - tmin) << 32 | e
        if (val) {  // carried by the sort
            const unsigned long long vv = val[x];
            e = (int32_t)(vv >> 32);
            tt = (int64_t)(vv & 0xffffffffull) + tmin;
            pk = (vv << 32) | (vv >> 32);
        } else {
            const TE rec = te[r];
            e = rec.e;
            tt = rec.t;
        }
        if (code & 1ull) {
            const int64_t slot = ob;
            out_t[slot] = tt;
            out_id[slot] = e;
            out_r[slot] = r;
            pos_out[e] = (int32_t)slot;
            // b: in-edges of v with t <= t_r; v's in-list starts at moff[v] - out_off[v]
            if (outrk) outrk[r] = make_int4((int32_t)slot, (int32_t)(seg - obv), (int32_t)(moff[v] - out_off[v]), 0);
            out_vb[slot] = make_int2((int32_t)v, (int32_t)(seg - obv));
            if (val) out_key[slot] = pk;
        } else {
            const int64_t slot = x - ob;
            in_t[slot] = tt;
            in_id[slot] = e;
            in_r[slot] = r;
            pos_in[e] = (int32_t)slot;
            in_head[slot] = (seg - obv) == 0;    // first entry of v's in-list
            if (inrk) inrk[r] = make_int2((int32_t)ob, (int32_t)out_off[v + 1]);  // ob = out_off[v] + a
            in_va[slot] = make_int2((int32_t)v, (int32_t)obv);
            if (val) in_key[slot] = pk;
        }
    }
}

// key ((t - tmin) << idbits | id), value (src, dst) in global vertex ids
__global__ void k_pack_keys(const int64_t *t, const int32_t *src, const int32_t *dst, const int32_t *egraph,
                            const int64_t *voff, int G, int64_t E, long long tmin, int idbits,
                            unsigned long long *k, unsigned long long *v) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        k[e] = ((unsigned long long)(t[e] - tmin) << idbits) | (unsigned long long)e;
        const int32_t vo = G > 1 ? (int32_t)voff[egraph[e]] : 0;
        v[e] = (unsigned long long)(unsigned)(src[e] + vo) | ((unsigned long long)(unsigned)(dst[e] + vo) << 32);
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

// off[v] = first sorted position whose vertex (key >> idbits) is >= v, for v in [0, V]
__global__ void k_voffsets(const unsigned long long *key, int64_t E, int64_t V, int idbits, int64_t *off) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= E;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = x < E ? (int64_t)(key[x] >> idbits) : V;
        const int64_t prev = x > 0 ? (int64_t)(key[x - 1] >> idbits) : -1;
        for (int64_t u = prev + 1; u <= v; u++) off[u] = x;
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
    o.outrk = ws.take<int4>(p.E);
    o.pos_out = ws.take<int32_t>(p.E);
    o.pos_in = ws.take<int32_t>(p.E);
    o.inrk = ws.take<int2>(p.E);
    o.in_gs = ws.take<int32_t>(p.E);
    o.in_va = ws.take<int2>(p.E);
    o.out_vb = ws.take<int2>(p.E);
    o.out_key = ws.take<unsigned long long>(p.E);
    o.in_key = ws.take<unsigned long long>(p.E);
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
    long long *flags;
    unsigned long long *mk, *mk2;  // [2E] incidence-item keys (the first sort uses both halves)
    unsigned long long *mv, *mv2;  // [2E] their values (original id, t - tmin) when the span fits 32 bits
    int *gflag;                    // [E+1] time-group heads
    long long *gpos, *scan_tmp;    // [E+1] group index (exclusive)
    int32_t *gstart;               // [E+1]
    int64_t *moff;                 // [V+1] merged-list offsets
    int32_t *oidx;                 // [2E+1] out-items before each item
    unsigned char *in_head;        // [E] first entry of an in-list
    TE *te;                        // [E] by r: (t, original id)
    void *radix;
};
static CsrScratch carve_csr(Arena &a, const Problem &p) {
    CsrScratch s;
    int64_t E = p.E > 0 ? p.E : 1;
    s.flags = a.take<long long>(8);
    s.mk = a.take<unsigned long long>(2 * E);
    s.mk2 = a.take<unsigned long long>(2 * E);
    s.mv = a.take<unsigned long long>(2 * E);
    s.mv2 = a.take<unsigned long long>(2 * E);
    s.gflag = a.take<int>(E + 1);
    s.gpos = a.take<long long>(E + 1);
    s.gstart = a.take<int32_t>(E + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(2 * E + 1));
    s.moff = a.take<int64_t>(p.V + 1);
    s.oidx = a.take<int32_t>(2 * E + 1);
    s.in_head = a.take<unsigned char>(E);
    s.te = a.take<TE>(E);
    s.radix = a.take<char>(radix_scratch_bytes(2 * E));
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
        TK(c, "k_hub_scatter", k_hub_scatter<<<grid_for(tot, kBlock, kStreamCap), kBlock, 0, st>>>(hub_of, key_of, tot, off, hl, hstart,
                                                                       keys));
    }
    return DGEC_OK;
}

// Scan loaders and stores for the merged lists.
struct LoadOutBit {  // 1 for an out-item, 0 for an in-item or past the end
    const unsigned long long *k;
    int64_t n;
    __device__ __forceinline__ long long operator()(int64_t i) const { return i < n ? (long long)(k[i] & 1ull) : 0ll; }
};
struct StoreI32 {
    int32_t *p;
    __device__ __forceinline__ void operator()(int64_t i, long long v) const { p[i] = (int32_t)v; }
};
// y where a time group starts in the in-lists (a list's first entry, or a
// time different from the entry before), 0 elsewhere: the running maximum
// is then the start of y's tie group.
struct LoadInGroupHead {
    const int64_t *t;
    const unsigned char *head;
    __device__ __forceinline__ long long operator()(int64_t y) const {
        return (head[y] || y == 0 || t[y] != t[y - 1]) ? (long long)y : 0ll;
    }
};
struct MaxI64 {
    __device__ __forceinline__ long long operator()(long long a, long long b) const { return a > b ? a : b; }
};

dgec_status stage_csr(Ctx *c, Problem &p, Csr &o, void *scratch) {
    cudaStream_t st = c->stream;
    Arena a(scratch, SIZE_MAX);
    CsrScratch s = carve_csr(a, p);
    int64_t V = p.V, E = p.E;
    TK(c, "k_init_flags", k_init_flags<<<1, 1, 0, st>>>(s.flags));
    if (E > 0) {
        if (p.G == 1) CU_TRY(c, cudaMemsetAsync(p.egraph, 0, sizeof(int32_t) * E, st));
        else TK(c, "k_egraph", k_egraph<<<grid_for(E, kBlock, kStreamCap), kBlock, 0, st>>>(p.eoff, p.G, E, p.egraph));
        TK(c, "k_count", k_count<<<grid_for(E, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                             p.src, p.dst, p.t, E, p.egraph, p.voff, nullptr, nullptr, s.flags));
    }
    int64_t f[4];
    DG_TRY(read_counters(c, (const int64_t *)s.flags, 4, f));
    if (f[0]) return set_err(c, DGEC_ERR_VERTEX_RANGE, "%lld edges have a vertex id outside their graph's range",
                             (long long)f[0]);
    if (f[1]) return set_err(c, DGEC_ERR_SELF_LOOP, "%lld self loops (i, i, t)", (long long)f[1]);
    p.tmin = E > 0 ? f[2] : 0;
    uint64_t span = E > 0 ? (uint64_t)f[3] - (uint64_t)f[2] : 0;
    p.idbits = bits_for((uint64_t)(E > 1 ? E - 1 : 1));
    p.tbits = bits_for(span);
    // forms 1 and 2 read packed keys, written only when every t - tmin fits 32 bits
    p.knn_form = p.tbits > 32 ? 0 : c->knn_packed;
    if (E == 0) {
        CU_TRY(c, cudaMemsetAsync(o.out_off, 0, sizeof(int64_t) * (V + 1), st));
        CU_TRY(c, cudaMemsetAsync(o.in_off, 0, sizeof(int64_t) * (V + 1), st));
        return DGEC_OK;
    }
    // global (t, id) order: internal ids
    const int gEE = grid_for(E, kBlock, kStreamCap);
    if (p.idbits + p.tbits <= 64) {
        TK(c, "k_pack_keys", k_pack_keys<<<gEE, kBlock, 0, st>>>(p.t, p.src, p.dst, p.egraph, p.voff, p.G, E, p.tmin,
                                                                p.idbits, s.mk, s.mk + E));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.mk, s.mk2, s.mk + E, s.mk2 + E}, E, p.idbits, p.idbits + p.tbits,
                          s.radix, &in_b));
        TK(c, "k_rank_init", k_rank_init<<<gEE, kBlock, 0, st>>>(in_b ? s.mk2 : s.mk, in_b ? s.mk2 + E : s.mk + E, E,
                                                                p.tmin, p.idbits, o.orig_of, o.rank_of, o.isrc, o.idst,
                                                                o.it, p.tbits <= 32 ? nullptr : s.te));
    } else {
        // wide span: the time is the whole key, the id its value (second halves of the item buffers)
        TK(c, "k_pack_t", k_pack_t<<<gEE, kBlock, 0, st>>>(p.t, E, p.tmin, s.mk, s.mk + E));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.mk, s.mk2, s.mk + E, s.mk2 + E}, E, 0, p.tbits, s.radix, &in_b));
        TK(c, "k_rank_init_kv", k_rank_init_kv<<<gEE, kBlock, 0, st>>>(
                                    in_b ? s.mk2 : s.mk, in_b ? s.mk2 + E : s.mk + E, E, p.tmin, p.src, p.dst,
                                    p.egraph, p.voff, p.G, o.orig_of, o.rank_of, o.isrc, o.idst, o.it, s.te));
    }
    // time groups of the r order, then the incidence items in (t, in-before-out, r) order
    TK(c, "k_thead", k_thead<<<grid_for(E + 1, kBlock, kStreamCap), kBlock, 0, st>>>(o.it, E, s.gflag));
    DG_TRY(exclusive_scan_i32(c, s.gflag, s.gpos, E + 1, s.scan_tmp));
    TK(c, "k_tgstart", k_tgstart<<<grid_for(E + 1, kBlock, kStreamCap), kBlock, 0, st>>>(s.gflag, s.gpos, E, s.gstart));
    const int cb = p.idbits + 1;  // bits of an item code 2r + dir
    const int vbits = bits_for((uint64_t)(V > 1 ? V - 1 : 1));
    const bool carry = p.tbits <= 32;  // (id, t - tmin) fits the 64-bit sort value
    TK(c, "k_mkeys", k_mkeys<<<gEE, kBlock, 0, st>>>(o.isrc, o.idst, s.gflag, s.gpos, s.gstart, E, cb, s.mk,
                                                     o.orig_of, o.it, p.tmin, carry ? s.mv : nullptr));
    // every vertex's merged list: a stable sort over the vertex bits alone
    bool in_b;
    DG_TRY(radix_sort(c, RadixBuffers{s.mk, s.mk2, carry ? s.mv : nullptr, carry ? s.mv2 : nullptr}, 2 * E, cb,
                      cb + vbits, s.radix, &in_b));
    const unsigned long long *key = in_b ? s.mk2 : s.mk;
    const unsigned long long *mval = carry ? (in_b ? s.mv2 : s.mv) : nullptr;
    TK(c, "k_voffsets", k_voffsets<<<grid_for(2 * E + 1, kBlock, kStreamCap), kBlock, 0, st>>>(key, 2 * E, V, cb, s.moff));
    DG_TRY((device_scan<long long, SumI64, LoadOutBit, StoreI32>(c, LoadOutBit{key, 2 * E}, StoreI32{s.oidx},
                                                                 2 * E + 1, SumI64{}, 0ll, false, s.scan_tmp)));
    TK(c, "k_moff_split", k_moff_split<<<grid_for(V + 1, kBlock, kStreamCap), kBlock, 0, st>>>(s.moff, s.oidx, V, o.out_off,
                                                                                        o.in_off));
    // the per-edge kNN forms read the window places by r; the list-order form and the skeleton do not
    const bool rk = p.knn && p.knn_form != 2;
    TK(c, "k_munpack", k_munpack<<<grid_for(2 * E, kBlock, kStreamCap), kBlock, 0, st>>>(
                           key, mval, p.tmin, 2 * E, cb, s.moff, s.oidx, o.out_off, s.te, o.out_t, o.out_id,
                           o.out_r, rk ? o.outrk : nullptr,
                           o.pos_out, o.in_t, o.in_id, o.in_r, o.pos_in, s.in_head, rk ? o.inrk : nullptr, o.in_va,
                           o.out_vb, o.out_key, o.in_key));
    // start of every in-list entry's tie group (the kNN window takes a crossing group's smallest ids)
    DG_TRY((device_scan<long long, MaxI64, LoadInGroupHead, StoreI32>(c, LoadInGroupHead{o.in_t, s.in_head},
                                                                      StoreI32{o.in_gs}, E, MaxI64{}, 0ll, true,
                                                                      s.scan_tmp)));
    return DGEC_OK;
}

}  // namespace dgec
