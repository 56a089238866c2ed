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

// All node ids below are internal ids r (see the stage A notes).
struct SkView {
    const int32_t *src, *dst;  // isrc, idst (by r)
    const int64_t *out_off, *in_off;
    const int32_t *out_id, *in_id;    // out_r, in_r
    const int32_t *orig_of;           // r -> original id
    const int32_t *pos_out, *pos_in;  // original id -> list slot
    const int2 *in_va, *out_vb;       // by slot: (vertex, a) of in-entries, (vertex, b) of out-entries
};

// Does Alg. 2 at vertex x emit the pair (in-edge pin, out-edge qout)? Only
// asked for a reciprocal pair at equal times, so its scattered reads are rare.
__device__ __forceinline__ bool emitted_at(const SkView &g, int x, int pin, int qout) {
    const int64_t ob = g.out_off[x];
    const int64_t a0 = ob + g.in_va[g.pos_in[g.orig_of[pin]]].y;  // pin's first out-edge of x not before it
    if (a0 < g.out_off[x + 1] && g.out_id[a0] == qout) return true;  // type 1
    const int64_t sq = g.pos_out[g.orig_of[qout]];
    if (sq > ob) {  // type 2
        const int b = g.out_vb[sq - 1].y;
        if (b >= 1 && g.in_id[g.in_off[x] + b - 1] == pin) return true;
    }
    return false;
}

// The links, walking the lists in order (with the time cutoff of Sec. 4.3
// only links with w <= dmax are kept: by Thm. 3 the kept links have, at
// every threshold, the components of the line graph without the longer
// arcs). Each link goes to a 16-byte record at its emitting edge's internal
// id (type 1 at r, type 2 at E + r), so the compacted skeleton keeps the
// (t, id) order of the emitting edges and the forest rounds read their
// endpoints with time locality; partner -1 where there is no link.
struct LinkRec {
    int32_t partner;
    int32_t keep;
    int64_t w;
};

// Type 1, over the in-list slots: the in-edge e at slot x of vertex j (its
// p_x) links to q_{a_x}, the first out-edge of j not before it. a is
// nondecreasing along j's in-list, so the partners are read nearly in order.
__global__ void k_links_in(SkView g, const int2 *in_va, const int64_t *out_t, const int64_t *in_t, int64_t E,
                           int64_t dmax, LinkRec *rec) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int2 va = in_va[x];
        const int j = va.x, a = va.y, e = g.in_id[x];
        const int64_t ob = g.out_off[j], nout = g.out_off[j + 1] - ob;
        LinkRec l{-1, 0, 0};
        if (a < nout) {
            const int q = g.out_id[ob + a];
            const int64_t w = out_t[ob + a] - in_t[x];
            // a reciprocal concurrent pair is kept once (at the vertex whose in-edge has the smaller id)
            const bool drop = (w == 0) && g.dst[q] == g.src[e] && e > q && emitted_at(g, g.src[e], q, e);
            if (!drop) l = LinkRec{q, w <= dmax, w};
        }
        rec[e] = l;
    }
}

// Type 2, over the out-list slots: the out-edge e at slot y of vertex i (its
// q_m, m >= 1) links to p_{b_{m-1} - 1}, where b_{m-1} is the b of the
// out-edge in slot y - 1; b is nondecreasing along i's out-list.
__global__ void k_links_out(SkView g, const int2 *out_vb, const int64_t *out_t, const int64_t *in_t,
                            int64_t E, int64_t dmax, LinkRec *rec) {
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < E;
         y += (int64_t)gridDim.x * blockDim.x) {
        const int i = out_vb[y].x, e = g.out_id[y];
        LinkRec l{-1, 0, 0};
        if (y > g.out_off[i]) {
            const int b = out_vb[y - 1].y;
            if (b >= 1) {
                const int64_t pp = g.in_off[i] + b - 1;
                const int p = g.in_id[pp];
                const int64_t w = out_t[y] - in_t[pp];
                const bool drop = (w == 0) && g.src[p] == g.dst[e] && p > e && emitted_at(g, g.dst[e], e, p);
                if (!drop) l = LinkRec{p, w <= dmax, w};
            }
        }
        rec[E + e] = l;
    }
}

struct LoadKeep {
    const LinkRec *rec;
    int64_t n;
    __device__ __forceinline__ long long operator()(int64_t i) const { return i < n ? rec[i].keep : 0; }
};

__global__ void k_compact_links(const LinkRec *rec, const long long *pos, int64_t E, const int32_t *orig_of,
                                int32_t *ru, int32_t *rv, int32_t *u, int32_t *v, int64_t *w) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < 2 * E;
         x += (int64_t)gridDim.x * blockDim.x) {
        const LinkRec l = rec[x];
        if (!l.keep) continue;
        const int self = (int)(x < E ? x : x - E), o = l.partner;
        const int es = orig_of[self], eo = orig_of[o];
        const int64_t at = pos[x];
        ru[at] = self;
        rv[at] = o;
        u[at] = es < eo ? es : eo;
        v[at] = es < eo ? eo : es;
        w[at] = l.w;
    }
}

// ---------------------------------------------------------------- kNN
// Neighbours of e = (i, j, t_e) in the undirected L_G: in-edges r of i with
// t_r <= t_e (prefix of i's in-list of length b[e]) and out-edges s of
// j with t_s >= t_e (suffix of j's out-list from its slot inrk[e].x). Ranked by
// (|dt|, id). The K best of each side suffice: the successor side is
// already in (w, id) order from its first slot; on the predecessor side the last K
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
__global__ void __launch_bounds__(256) k_knn(const int64_t *t, const int32_t *orig_of, int64_t E,
                                             const int64_t *out_t, const int32_t *out_id,
                                             const int64_t *in_t, const int32_t *in_id,
                                             const int32_t *in_gs, const int4 *outrk, const int2 *inrk,
                                             int G,
                                             const int32_t *egraph, const int64_t *eoff,
                                             const int32_t *gk, const int64_t *knn_off, int64_t dmax,
                                             int32_t *knn, int64_t *core) {
    constexpr int N = 2 * K;
    // r runs over internal ids (src, dst, t are the r-ordered copies); the
    // neighbour lists are written under the original id, with original ids
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const long long te = t[r];
        const int64_t e = orig_of[r];
        // the edge's graph: its k, its kNN rows, its local id base
        const int gr = G > 1 ? egraph[e] : 0;  // one graph: no random lookup
        const int k = gk[gr];
        const int64_t e0 = eoff[gr];
        int32_t *row = knn + knn_off[gr] + (e - e0) * k;
        // the two windows' places come with the edge: no offset lookups
        const int4 orec = outrk[r];
        const int2 irec = inrk[r];
        const int64_t b = orec.y, ib = orec.z;
        const int64_t a0 = irec.x, a1 = irec.y;  // successor window: out-list slots [a0, a1)
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
            const int64_t idx = a0 + x;
            if (idx < a1) {
                c[K + x].w = out_t[idx] - te;
                c[K + x].id = out_id[idx];
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

// The same for time spans below 2^32 (every |dt| fits 32 bits): each list
// entry is one 64-bit key ((t - tmin) << 32 | id) written by stage A, so a
// window is one run of one array (half the sectors of separate time and id
// arrays), and a candidate is one 64-bit key (w << 32 | id): the network
// sorts plain integers (two registers a candidate instead of three, one
// compare a step) and the kernel keeps more warps resident to hide its
// gathers' latency.
template <int K>
__global__ void __launch_bounds__(256, K <= 8 ? 3 : 1) k_knn32(const int64_t *t, long long tmin,
                                               const int32_t *orig_of, int64_t E,
                                               const unsigned long long *__restrict__ out_key,
                                               const unsigned long long *__restrict__ in_key,
                                               const int32_t *in_gs, const int4 *outrk, const int2 *inrk,
                                               int G,
                                               const int32_t *egraph, const int64_t *eoff,
                                               const int32_t *gk, const int64_t *knn_off, int64_t dmax,
                                               int32_t *knn, int64_t *core) {
    constexpr int N = 2 * K;
    constexpr unsigned long long kNone = 0xFFFFFFFFFFFFFFFFull;
    constexpr unsigned long long kLo = 0xFFFFFFFFull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long te = (unsigned long long)(t[r] - tmin);
        const int64_t e = orig_of[r];
        const int gr = G > 1 ? egraph[e] : 0;
        const int k = gk[gr];
        const int64_t e0 = eoff[gr];
        int32_t *row = knn + knn_off[gr] + (e - e0) * k;
        // the two windows' places come with the edge: no offset lookups
        const int4 orec = outrk[r];
        const int2 irec = inrk[r];
        const int64_t b = orec.y, ib = orec.z;
        const int64_t a0 = irec.x, a1 = irec.y;  // successor window: out-list slots [a0, a1)
        unsigned long long c[N];
        const int64_t lo = b - K > 0 ? b - K : 0;
        int64_t g0 = lo, take_grp = 0;
        const unsigned long long tlo = lo < b ? in_key[ib + lo] >> 32 : 0;
        const bool cross = lo > 0 && tlo == (in_key[ib + lo - 1] >> 32);
        if (cross) {
            g0 = (int64_t)in_gs[ib + lo] - ib;
            int64_t g1 = lo;
            while (g1 < b && (in_key[ib + g1] >> 32) == tlo) g1++;  // at most K steps
            take_grp = g1 - lo;
        }
#pragma unroll
        for (int x = 0; x < K; x++) {
            const int64_t idx = x < take_grp ? g0 + x : lo + x;
            if (idx < b) {
                const unsigned long long kk = in_key[ib + idx];
                c[x] = ((te - (kk >> 32)) << 32) | (kk & kLo);
            } else {
                c[x] = kNone;
            }
        }
#pragma unroll
        for (int x = 0; x < K; x++) {
            const int64_t idx = a0 + x;
            if (idx < a1) {
                const unsigned long long kk = out_key[idx];
                c[K + x] = (((kk >> 32) - te) << 32) | (kk & kLo);
            } else {
                c[K + x] = kNone;
            }
        }
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
                for (int lo2 = 0; lo2 < N; lo2++) {
                    const int hi2 = lo2 ^ stride;
                    if (hi2 > lo2) {
                        const bool up = (lo2 & size) == 0;
                        const unsigned long long x0 = c[lo2], x1 = c[hi2];
                        const bool sw = up ? x1 < x0 : x0 < x1;
                        c[lo2] = sw ? x1 : x0;
                        c[hi2] = sw ? x0 : x1;
                    }
                }
            }
        }
        int cnt = 0;
        long long last_w = LLONG_MAX;
        unsigned prev = 0xFFFFFFFFu;
#pragma unroll
        for (int x = 0; x < N; x++) {
            const unsigned id = (unsigned)c[x];
            const long long w = (long long)(c[x] >> 32);
            if (c[x] != kNone && id != prev && cnt < k && w <= dmax) {
                row[cnt] = (int32_t)((int64_t)id - e0);
                last_w = w;
                cnt++;
            }
            prev = id;
        }
        for (int x = cnt; x < k; x++) row[x] = -1;
        core[e] = cnt == k ? last_w : LLONG_MAX;
    }
}

// The same candidates and selection in list order, as two passes that read
// their windows nearly in sequence. An edge e = (i, j, t) has its
// predecessors in i's in-list, before e's place among i's out-items, and its
// successors in j's out-list, after e's place among j's in-items. Walking
// the out-lists slot by slot, consecutive slots of one vertex read
// overlapping predecessor windows; walking the in-lists slot by slot, the
// same holds for the successor windows. So:
//   pass 1 (out-list slots): e's K predecessor keys, stored as one 8K-byte
//          run at e's in-list slot (one scattered 4-byte read of that slot
//          and whole-sector scattered writes; no load waits on another);
//   pass 2 (in-list slots): e's K successor keys, its predecessor keys read
//          in sequence from its own slot, the 2K-candidate sort and the row.
// The per-edge form above reads both windows at scattered places, several
// sectors each, and its warps wait on them.
template <int K>
__global__ void __launch_bounds__(256) k_knn_pred(int64_t E, const unsigned long long *__restrict__ out_key,
                                                  const int2 *__restrict__ out_vb,
                                                  const int64_t *__restrict__ in_off,
                                                  const unsigned long long *__restrict__ in_key,
                                                  const int32_t *__restrict__ in_gs,
                                                  const int32_t *__restrict__ pos_in,
                                                  ulonglong2 *__restrict__ half) {
    constexpr unsigned long long kNone = 0xFFFFFFFFFFFFFFFFull;
    constexpr unsigned long long kLo = 0xFFFFFFFFull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long q = out_key[x];
        const int2 vb = out_vb[x];
        const int32_t y = pos_in[(int64_t)(q & kLo)];  // e's in-list slot: where pass 2 reads its keys
        const unsigned long long te = q >> 32;
        const int64_t ib = in_off[vb.x], b = vb.y;
        unsigned long long c[K];
        const int64_t lo = b - K > 0 ? b - K : 0;
        int64_t g0 = lo, take_grp = 0;
        const unsigned long long tlo = lo < b ? in_key[ib + lo] >> 32 : 0;
        const bool cross = lo > 0 && tlo == (in_key[ib + lo - 1] >> 32);
        if (cross) {  // a tie group crossing the window's start gives its smallest ids
            g0 = (int64_t)in_gs[ib + lo] - ib;
            int64_t g1 = lo;
            while (g1 < b && (in_key[ib + g1] >> 32) == tlo) g1++;  // at most K steps
            take_grp = g1 - lo;
        }
#pragma unroll
        for (int u = 0; u < K; u++) {
            const int64_t idx = u < take_grp ? g0 + u : lo + u;
            if (idx < b) {
                const unsigned long long kk = in_key[ib + idx];
                c[u] = ((te - (kk >> 32)) << 32) | (kk & kLo);
            } else {
                c[u] = kNone;
            }
        }
        ulonglong2 *dstp = half + (int64_t)y * (K / 2);
#pragma unroll
        for (int u = 0; u < K / 2; u++) dstp[u] = make_ulonglong2(c[2 * u], c[2 * u + 1]);
    }
}

template <int K>
__global__ void __launch_bounds__(256, K <= 8 ? 3 : 1) k_knn_succ(
    int64_t E, const unsigned long long *__restrict__ in_key, const int2 *__restrict__ in_va,
    const int64_t *__restrict__ out_off, const unsigned long long *__restrict__ out_key,
    const ulonglong2 *__restrict__ half, int G, const int32_t *egraph, const int64_t *eoff,
    const int32_t *gk, const int64_t *knn_off, int64_t dmax, int32_t *knn, int64_t *core) {
    constexpr int N = 2 * K;
    constexpr unsigned long long kNone = 0xFFFFFFFFFFFFFFFFull;
    constexpr unsigned long long kLo = 0xFFFFFFFFull;
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < E;
         y += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long p = in_key[y];
        const int2 va = in_va[y];
        const unsigned long long te = p >> 32;
        const int64_t e = (int64_t)(p & kLo);
        const int64_t a0 = out_off[va.x] + va.y, a1 = out_off[va.x + 1];  // successor window [a0, a1)
        unsigned long long c[N];
        const ulonglong2 *srcp = half + y * (K / 2);
#pragma unroll
        for (int u = 0; u < K / 2; u++) {
            const ulonglong2 h = srcp[u];
            c[2 * u] = h.x;
            c[2 * u + 1] = h.y;
        }
#pragma unroll
        for (int u = 0; u < K; u++) {
            const int64_t idx = a0 + u;
            if (idx < a1) {
                const unsigned long long kk = out_key[idx];
                c[K + u] = (((kk >> 32) - te) << 32) | (kk & kLo);
            } else {
                c[K + u] = kNone;
            }
        }
        const int gr = G > 1 ? egraph[e] : 0;
        const int k = gk[gr];
        const int64_t e0 = eoff[gr];
        int32_t *row = knn + knn_off[gr] + (e - e0) * k;
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
                for (int lo2 = 0; lo2 < N; lo2++) {
                    const int hi2 = lo2 ^ stride;
                    if (hi2 > lo2) {
                        const bool up = (lo2 & size) == 0;
                        const unsigned long long x0 = c[lo2], x1 = c[hi2];
                        const bool sw = up ? x1 < x0 : x0 < x1;
                        c[lo2] = sw ? x1 : x0;
                        c[hi2] = sw ? x0 : x1;
                    }
                }
            }
        }
        int cnt = 0;
        long long last_w = LLONG_MAX;
        unsigned prev = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < N; u++) {
            const unsigned id = (unsigned)c[u];
            const long long w = (long long)(c[u] >> 32);
            if (c[u] != kNone && id != prev && cnt < k && w <= dmax) {
                row[cnt] = (int32_t)((int64_t)id - e0);
                last_w = w;
                cnt++;
            }
            prev = id;
        }
        for (int u = cnt; u < k; u++) row[u] = -1;
        core[e] = cnt == k ? last_w : LLONG_MAX;
    }
}

// K of the kNN kernels: the batch's largest k rounded up to 4, 8 or 16
static int knn_kpad(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : 16); }

void plan_skel(Arena &ws, const Problem &p, Skel &o) {
    o.u = ws.take<int32_t>(2 * p.E);
    o.v = ws.take<int32_t>(2 * p.E);
    o.ru = ws.take<int32_t>(2 * p.E);
    o.rv = ws.take<int32_t>(2 * p.E);
    o.w = ws.take<int64_t>(2 * p.E);
    o.knn = p.knn ? ws.take<int32_t>(p.E * (int64_t)p.k) : nullptr;  // p.k: the largest k of the batch
    o.core = p.knn ? ws.take<int64_t>(p.E) : nullptr;
}

struct SkScratch {
    LinkRec *rec;
    long long *pos, *scan_tmp;
    ulonglong2 *half;  // list-order kNN: K predecessor keys per in-list slot
};
static SkScratch carve_skel(Arena &a, const Problem &p) {
    SkScratch s;
    s.rec = a.take<LinkRec>(2 * p.E);
    s.pos = a.take<long long>(2 * p.E + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(2 * p.E + 1));
    s.half = p.knn ? a.take<ulonglong2>(p.E * (int64_t)(knn_kpad(p.k) / 2)) : nullptr;
    return s;
}
size_t skel_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_skel(a, p);
    return a.off;
}

dgec_status stage_skeleton(Ctx *c, const Problem &p, const Csr &g, Skel &o, void *scratch) {
    cudaStream_t st = c->stream;
    o.n = 0;
    if (p.E == 0) return DGEC_OK;
    Arena a(scratch, SIZE_MAX);
    SkScratch s = carve_skel(a, p);
    int64_t E = p.E;
    const int kb = c->knn_block;
    int grid = grid_for(E, kb, 1 << 20);
#define KNN_ARGS                                                                                   \
    g.it, g.orig_of, E, g.out_t, g.out_id, g.in_t, g.in_id, g.in_gs, g.outrk, g.inrk, p.G, p.egraph, p.eoff, \
        p.gk, p.knn_off, p.dmax, o.knn, o.core
#define KNN32_ARGS                                                                                 \
    g.it, p.tmin, g.orig_of, E, g.out_key, g.in_key, g.in_gs, g.outrk, g.inrk, p.G, p.egraph, p.eoff, p.gk, \
        p.knn_off, p.dmax, o.knn, o.core
    if (p.knn && p.knn_form == 2) {  // packed keys, in list order (two passes)
        const int gl = grid_for(E, kb, 1 << 20);
#define KNN_PRED_ARGS E, g.out_key, g.out_vb, g.in_off, g.in_key, g.in_gs, g.pos_in, s.half
#define KNN_SUCC_ARGS \
    E, g.in_key, g.in_va, g.out_off, g.out_key, s.half, p.G, p.egraph, p.eoff, p.gk, p.knn_off, p.dmax, o.knn, o.core
        switch (knn_kpad(p.k)) {
        case 4:
            TK(c, "k_knn_pred", k_knn_pred<4><<<gl, kb, 0, st>>>(KNN_PRED_ARGS));
            TK(c, "k_knn", k_knn_succ<4><<<gl, kb, 0, st>>>(KNN_SUCC_ARGS));
            break;
        case 8:
            TK(c, "k_knn_pred", k_knn_pred<8><<<gl, kb, 0, st>>>(KNN_PRED_ARGS));
            TK(c, "k_knn", k_knn_succ<8><<<gl, kb, 0, st>>>(KNN_SUCC_ARGS));
            break;
        default:
            TK(c, "k_knn_pred", k_knn_pred<16><<<gl, kb, 0, st>>>(KNN_PRED_ARGS));
            TK(c, "k_knn", k_knn_succ<16><<<gl, kb, 0, st>>>(KNN_SUCC_ARGS));
            break;
        }
#undef KNN_PRED_ARGS
#undef KNN_SUCC_ARGS
    } else if (p.knn && p.knn_form == 1) {  // every |dt| fits 32 bits: packed list and candidate keys
        if (p.k <= 4) TK(c, "k_knn", k_knn32<4><<<grid, kb, 0, st>>>(KNN32_ARGS));
        else if (p.k <= 8) TK(c, "k_knn", k_knn32<8><<<grid, kb, 0, st>>>(KNN32_ARGS));
        else TK(c, "k_knn", k_knn32<16><<<grid, kb, 0, st>>>(KNN32_ARGS));
    } else if (p.knn) {
        if (p.k <= 4) TK(c, "k_knn", k_knn<4><<<grid, kb, 0, st>>>(KNN_ARGS));
        else if (p.k <= 8) TK(c, "k_knn", k_knn<8><<<grid, kb, 0, st>>>(KNN_ARGS));
        else TK(c, "k_knn", k_knn<16><<<grid, kb, 0, st>>>(KNN_ARGS));
    }
#undef KNN_ARGS
#undef KNN32_ARGS
    SkView v{g.isrc, g.idst, g.out_off, g.in_off, g.out_r, g.in_r, g.orig_of, g.pos_out, g.pos_in, g.in_va, g.out_vb};
    TK(c, "k_links_in", k_links_in<<<grid_for(E, kBlock, kStreamCap), kBlock, 0, st>>>(
                            v, g.in_va, g.out_t, g.in_t, E, p.dmax, s.rec));
    TK(c, "k_links_out", k_links_out<<<grid_for(E, kBlock, kStreamCap), kBlock, 0, st>>>(
                             v, g.out_vb, g.out_t, g.in_t, E, p.dmax, s.rec));
    DG_TRY((device_scan<long long, SumI64, LoadKeep, StorePtr<long long>>(
        c, LoadKeep{s.rec, 2 * E}, StorePtr<long long>{s.pos}, 2 * E + 1, SumI64{}, 0ll, false, s.scan_tmp)));
    TK(c, "k_compact_links", k_compact_links<<<grid_for(2 * E, kBlock, kStreamCap), kBlock, 0, st>>>(
                                 s.rec, s.pos, E, g.orig_of, o.ru, o.rv, o.u, o.v, o.w));
    int64_t n;
    DG_TRY(read_counters(c, (const int64_t *)(s.pos + 2 * E), 1, &n));
    o.n = n;
    return DGEC_OK;
}

}  // namespace dgec
