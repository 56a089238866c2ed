// Stage B: the line-graph skeleton L*_G (Alg. 2 per vertex, Alg. 3 union)
// and the k nearest line-graph neighbours in time.
//
// Alg. 2 as rank arithmetic. At vertex i, with in-edges p_0..p_{n-1} and
// out-edges q_0..q_{m-1} each sorted by (t, id), and in-edges ordered before
// out-edges at equal t, let b_m = #{x : t(p_x) <= t(q_m)}. When the sweep
// reaches q_m its buffer W holds p_x for x in [max(b_{m-1} - 1, 0), b_m)
// (b_{-1} = 0), so every emitted line-graph edge is one of:
//   type 1: each in-edge p_x with a later out-edge links to the first one,
//           q_{a_x}, a_x = #{m : t(q_m) < t(p_x)};
//   type 2: each out-edge q_m, m >= 1, links to the retained in-edge
//           p_{b_{m-1} - 1} when b_{m-1} >= 1.
// So each edge emits at most one type-1 link (at its destination) and one
// type-2 link (at its source): one thread per edge, no load imbalance on
// hubs, and |L*| <= sum_i (|E_i| - 1) (Sec. 2) falls out directly.
//
// The union of Alg. 3 is a set: a pair emitted at two vertices is a
// reciprocal, concurrent pair (i, j, t), (j, i, t) with w = 0; it is kept
// at the vertex whose in-edge has the smaller id.
#include "stages.cuh"

namespace dgec {

// brank[e] = #in-edges of src[e] with t <= t_e; arank[e] = #out-edges of
// dst[e] with t < t_e (both from stage A's merged lists).
// All node ids below are internal ids r (see the stage A notes).
struct SkView {
    const int32_t *src, *dst;  // isrc, idst (by r)
    const int64_t *out_off, *in_off;
    const int32_t *out_id, *in_id, *slot_out;  // out_r, in_r, slot_out (by r)
    const int32_t *brank, *arank;
};

// Does Alg. 2 at vertex x emit the pair (in-edge pin, out-edge qout)?
__device__ __forceinline__ bool emitted_at(const SkView &g, int x, int pin, int qout) {
    int64_t ob = g.out_off[x], nout = g.out_off[x + 1] - ob;
    int a = g.arank[pin];
    if (a < nout && g.out_id[ob + a] == qout) return true;  // type 1
    int64_t sq = g.slot_out[qout];
    if (sq > ob) {                                          // type 2
        int b = g.brank[g.out_id[sq - 1]];
        if (b >= 1 && g.in_id[g.in_off[x] + b - 1] == pin) return true;
    }
    return false;
}

// part[e] / part[E + e]: partner of edge e through its type-1 / type-2
// link (-1 if none), wgt the P3 weight. With the time cutoff of Sec. 4.3
// only links with w <= dmax are kept: by Thm. 3 the kept links have, at
// every threshold, the components of the line graph without the longer
// arcs.
__global__ void k_links(SkView g, const int64_t *t, const int64_t *out_t, const int64_t *in_t,
                        int64_t E, int64_t dmax, int32_t *part, int64_t *wgt, int *flag) {
    // e below is an internal id r; t, src, dst are the r-ordered copies
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = g.src[e], j = g.dst[e];
        int64_t te = t[e];
        // type 1: e is p_x at j, linked to q_{a_x}
        int32_t p1 = -1;
        int64_t w1 = 0;
        {
            int64_t ob = g.out_off[j], nout = g.out_off[j + 1] - ob;
            int a = g.arank[e];
            if (a < nout) {
                int q = g.out_id[ob + a];
                int64_t w = out_t[ob + a] - te;
                bool drop = (w == 0) && g.dst[q] == i && (int)e > q && emitted_at(g, i, q, (int)e);
                if (!drop) {
                    p1 = q;
                    w1 = w;
                }
            }
        }
        // type 2: e is q_m (m >= 1) at i, linked to p_{b_{m-1} - 1}
        int32_t p2 = -1;
        int64_t w2 = 0;
        {
            int64_t sl = g.slot_out[e];
            if (sl > g.out_off[i]) {
                int b = g.brank[g.out_id[sl - 1]];
                if (b >= 1) {
                    int64_t pp = g.in_off[i] + b - 1;
                    int p = g.in_id[pp];
                    int64_t w = te - in_t[pp];
                    bool drop = (w == 0) && g.src[p] == j && p > (int)e && emitted_at(g, j, (int)e, p);
                    if (!drop) {
                        p2 = p;
                        w2 = w;
                    }
                }
            }
        }
        part[e] = p1;
        wgt[e] = w1;
        part[E + e] = p2;
        wgt[E + e] = w2;
        flag[e] = p1 >= 0 && w1 <= dmax;
        flag[E + e] = p2 >= 0 && w2 <= dmax;
    }
}

__global__ void k_compact_links(const int32_t *part, const int64_t *wgt, const int *flag,
                                const long long *pos, int64_t E, const int32_t *orig_of, int32_t *ru,
                                int32_t *rv, int32_t *u, int32_t *v, int64_t *w) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < 2 * E;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[x]) continue;
        int self = (int)(x < E ? x : x - E), o = part[x];
        int64_t at = pos[x];
        int es = orig_of[self], eo = orig_of[o];
        ru[at] = self;
        rv[at] = o;
        u[at] = es < eo ? es : eo;
        v[at] = es < eo ? eo : es;
        w[at] = wgt[x];
    }
}

// ---------------------------------------------------------------- kNN
// Neighbours of e = (i, j, t_e) in the undirected L_G: in-edges r of i with
// t_r <= t_e (prefix of i's in-list of length brank[e]) and out-edges s of
// j with t_s >= t_e (suffix of j's out-list from arank[e]). Ranked by
// (|dt|, id). The K best of each side suffice: the successor side is
// already in (w, id) order from arank; on the predecessor side the last K
// of the prefix, except that when the boundary tie group crosses the
// window its smallest ids are taken instead of its largest (the group's
// first slot comes from stage A's in_gs). The two ranks come from stage A,
// so the kernel only gathers two windows of K contiguous entries: no
// search. The 2K candidates are sorted in registers (bitonic network); the
// one node that can appear on both sides (the reciprocal concurrent edge,
// w = 0) is counted once. Under the time cutoff (Sec. 4.3) only neighbours
// with w <= dmax exist; they are a prefix of the sorted candidates.

struct Cand {
    long long w;
    int id;
};
__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b) {
    return a.w < b.w || (a.w == b.w && a.id < b.id);
}

template <int K>
__global__ void __launch_bounds__(256) k_knn(const int32_t *src, const int32_t *dst, const int64_t *t,
                                             const int32_t *orig_of, int64_t E, const int64_t *out_off,
                                             const int64_t *out_t, const int32_t *out_id,
                                             const int64_t *in_off, const int64_t *in_t,
                                             const int32_t *in_id, const int32_t *in_gs,
                                             const int32_t *brank, const int32_t *arank, int G,
                                             const int32_t *egraph, const int64_t *eoff,
                                             const int32_t *gk, const int64_t *knn_off, int64_t dmax,
                                             int32_t *knn, int64_t *core) {
    constexpr int N = 2 * K;
    // r runs over internal ids (src, dst, t are the r-ordered copies); the
    // neighbour lists are written under the original id, with original ids
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int i = src[r], j = dst[r];
        const long long te = t[r];
        const int64_t e = orig_of[r];
        // the edge's graph: its k, its kNN rows, its local id base
        const int gr = G > 1 ? egraph[e] : 0;  // one graph: no random lookup
        const int k = gk[gr];
        const int64_t e0 = eoff[gr];
        int32_t *row = knn + knn_off[gr] + (e - e0) * k;
        const int64_t ib = in_off[i];
        const int64_t ob = out_off[j], nout = out_off[j + 1] - ob;
        const int64_t b = brank[r], a = arank[r];
        Cand c[N];
        // predecessor window: the last K of the prefix [0, b); a tie group
        // that crosses its start contributes its smallest ids
        const int64_t lo = b - K > 0 ? b - K : 0;
        int64_t g0 = lo, take_grp = 0;
        const bool cross = lo > 0 && in_t[ib + lo] == in_t[ib + lo - 1];
        if (cross) {
            const long long T = in_t[ib + lo];
            g0 = (int64_t)in_gs[ib + lo] - ib;
            int64_t g1 = lo;
            while (g1 < b && in_t[ib + g1] == T) g1++;  // at most K steps
            take_grp = g1 - lo;
        }
#pragma unroll
        for (int x = 0; x < K; x++) {
            const int64_t idx = x < take_grp ? g0 + x : lo + x;
            if (idx < b) {
                c[x].w = te - in_t[ib + idx];
                c[x].id = in_id[ib + idx];
            } else {
                c[x].w = LLONG_MAX;
                c[x].id = INT_MAX;
            }
        }
#pragma unroll
        for (int x = 0; x < K; x++) {
            const int64_t idx = a + x;
            if (idx < nout) {
                c[K + x].w = out_t[ob + idx] - te;
                c[K + x].id = out_id[ob + idx];
            } else {
                c[K + x].w = LLONG_MAX;
                c[K + x].id = INT_MAX;
            }
        }
        // bitonic sort of N candidates, ascending by (w, id)
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
                for (int lo2 = 0; lo2 < N; lo2++) {
                    int hi2 = lo2 ^ stride;
                    if (hi2 > lo2) {
                        bool up = (lo2 & size) == 0;
                        bool sw = up ? cand_less(c[hi2], c[lo2]) : cand_less(c[lo2], c[hi2]);
                        if (sw) {
                            Cand tmp = c[lo2];
                            c[lo2] = c[hi2];
                            c[hi2] = tmp;
                        }
                    }
                }
            }
        }
        int cnt = 0;
        long long last_w = LLONG_MAX;
        int prev = -1;
#pragma unroll
        for (int x = 0; x < N; x++) {
            if (c[x].id != INT_MAX && c[x].id != prev && cnt < k && c[x].w <= dmax) {
                row[cnt] = (int32_t)(c[x].id - e0);
                last_w = c[x].w;
                cnt++;
            }
            prev = c[x].id;
        }
        for (int x = cnt; x < k; x++) row[x] = -1;
        core[e] = cnt == k ? last_w : LLONG_MAX;
    }
}

void plan_skel(Arena &ws, const Problem &p, Skel &o) {
    o.brank = o.arank = nullptr;  // the ranks live in stage A's output
    o.u = ws.take<int32_t>(2 * p.E);
    o.v = ws.take<int32_t>(2 * p.E);
    o.ru = ws.take<int32_t>(2 * p.E);
    o.rv = ws.take<int32_t>(2 * p.E);
    o.w = ws.take<int64_t>(2 * p.E);
    o.knn = p.knn ? ws.take<int32_t>(p.E * (int64_t)p.k) : nullptr;  // p.k: the largest k of the batch
    o.core = p.knn ? ws.take<int64_t>(p.E) : nullptr;
}

struct SkScratch {
    int32_t *part;
    int64_t *wgt;
    int *flag;
    long long *pos, *scan_tmp;
};
static SkScratch carve_skel(Arena &a, const Problem &p) {
    SkScratch s;
    s.part = a.take<int32_t>(2 * p.E);
    s.wgt = a.take<int64_t>(2 * p.E);
    s.flag = a.take<int>(2 * p.E + 1);
    s.pos = a.take<long long>(2 * p.E + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(2 * p.E + 1));
    return s;
}
size_t skel_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_skel(a, p);
    return a.off;
}

__global__ void k_zero_i32(int *p) { *p = 0; }

dgec_status stage_skeleton(Ctx *c, const Problem &p, const Csr &g, Skel &o, void *scratch) {
    cudaStream_t st = c->stream;
    o.n = 0;
    if (p.E == 0) return DGEC_OK;
    Arena a(scratch, SIZE_MAX);
    SkScratch s = carve_skel(a, p);
    int64_t E = p.E;
    const int kb = c->knn_block;
    int grid = grid_for(E, kb, 1 << 20);
    o.brank = g.brank;
    o.arank = g.arank;
#define KNN_ARGS                                                                                   \
    g.isrc, g.idst, g.it, g.orig_of, E, g.out_off, g.out_t, g.out_id, g.in_off, g.in_t, g.in_id, g.in_gs, \
        g.brank, g.arank, p.G, p.egraph, p.eoff, p.gk, p.knn_off, p.dmax, o.knn, o.core
    if (p.knn) {
        if (p.k <= 4) TK(c, "k_knn", k_knn<4><<<grid, kb, 0, st>>>(KNN_ARGS));
        else if (p.k <= 8) TK(c, "k_knn", k_knn<8><<<grid, kb, 0, st>>>(KNN_ARGS));
        else TK(c, "k_knn", k_knn<16><<<grid, kb, 0, st>>>(KNN_ARGS));
    }
#undef KNN_ARGS
    SkView v{g.isrc, g.idst, g.out_off, g.in_off, g.out_r, g.in_r, g.slot_out, o.brank, o.arank};
    TK(c, "k_links", k_links<<<grid_for(E, kBlock, kStreamCap), kBlock, 0, st>>>(v, g.it, g.out_t, g.in_t, E, p.dmax,
                                                                          s.part, s.wgt, s.flag));
    TK(c, "k_zero_i32", k_zero_i32<<<1, 1, 0, st>>>(s.flag + 2 * E));
    DG_TRY(exclusive_scan_i32(c, s.flag, s.pos, 2 * E + 1, s.scan_tmp));
    TK(c, "k_compact_links", k_compact_links<<<grid_for(2 * E, kBlock, kStreamCap), kBlock, 0, st>>>(
                                 s.part, s.wgt, s.flag, s.pos, E, g.orig_of, o.ru, o.rv, o.u, o.v, o.w));
    int64_t n;
    DG_TRY(read_counters(c, (const int64_t *)(s.pos + 2 * E), 1, &n));
    o.n = n;
    return DGEC_OK;
}

}  // namespace dgec
