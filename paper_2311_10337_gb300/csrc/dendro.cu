// Stage D1: single-linkage dendrogram (Alg. 1, union-find dendrogram) of the sorted
// forest, built in parallel rounds instead of one union-find sweep.
//
// Merge s is the s-th forest edge in (w, u, v) order; its dendrogram node is
// n_edges + s. Every round works on the super-vertices (already merged
// subtrees) and the forest edges not yet placed:
//   1. each super-vertex takes its smallest incident edge (its "pointer");
//      pointers form trees whose root is the one mutual pair, and along a
//      pointer path the edge ranks decrease toward that pair;
//   2. tau(G) = smallest non-pointer edge touching pointer tree G;
//   3. the pointer edges of G below tau(G) are accepted. They form a
//      connected top part of G, and no other edge below them touches it, so
//      in rank order g_1 < g_2 < ... they merge as a chain: g_1 joins the
//      mutual pair's two subtrees, g_k joins g_{k-1} with the subtree of the
//      super-vertex whose pointer g_k is;
//   4. sizes along a chain are a segmented prefix sum; the accepted part of
//      G becomes one super-vertex whose dendrogram root is its last merge.
// Each round accepts at least the mutual edge of every pointer tree, and a
// pointer tree with no interfering edge is placed whole (a star is one
// round), so the round count follows the depth of interference, not the
// dendrogram height.
#include "stages.cuh"

namespace dgec {

// Super-vertex labels are internal ids r (a leaf's label is its own r).
// Each super-vertex's dendrogram root (a node id, so a leaf's root is its
// original id) and size share one 16-byte record: a chain step reads both
// with one sector.
struct SvRec {
    int64_t size;
    int32_t root;
    int32_t pad;
};
//
// minr (a super-vertex's smallest live edge) and tau (a pointer tree's
// smallest non-pointer edge) live one round each. A slot holds
// (stamp << 32) | rank with stamp = kStampTop - round: newer rounds have
// smaller stamps, so atomicMin over the whole key keeps this round's
// minimum, and a slot with another stamp holds nothing this round. No pass
// resets them between rounds.
constexpr unsigned kStampTop = 0xFFFFFFF0u;
__device__ __forceinline__ unsigned long long rkey(unsigned stamp, int v) {
    return ((unsigned long long)stamp << 32) | (unsigned)v;
}
__device__ __forceinline__ int rval(unsigned long long k, unsigned stamp) {
    return (unsigned)(k >> 32) == stamp ? (int)(unsigned)k : INT_MAX;
}
__global__ void k_d_init(int64_t E, int64_t n, const int32_t *mu, const int32_t *mv,
                         const int32_t *orig_of, int32_t *svpar, SvRec *sv,
                         unsigned long long *minr, unsigned long long *tau, int32_t *parent, int32_t *act, int32_t *ecu,
                         int32_t *ecv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E + n;
         x += (int64_t)gridDim.x * blockDim.x) {
        parent[x] = -1;
        if (x < E) {
            svpar[x] = (int32_t)x;
            sv[x] = SvRec{1, orig_of[x], 0};
            minr[x] = ~0ull;
            tau[x] = ~0ull;
        }
        if (x < n) {
            act[x] = (int32_t)x;
            ecu[x] = mu[x];
            ecv[x] = mv[x];
        }
    }
}

// Every live forest edge bids its rank into the super-vertices at its ends.
// The labels (ecu, ecv) travel with the edge and are moved one hop after
// each round's merges, so no label chain is ever walked. A read before the
// atomic skips bids that cannot win (slots only decrease).
__global__ void k_d_bid(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                        unsigned long long *minr, unsigned stamp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        int s = act[j];
        int cu = ecu[j], cv = ecv[j];
        const unsigned long long key = rkey(stamp, s);
        if (key < minr[cu]) atomicMin(&minr[cu], key);
        if (key < minr[cv]) atomicMin(&minr[cv], key);
    }
}

__global__ void k_d_ptr(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                        const unsigned long long *minr, unsigned stamp, int32_t *gp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        int s = act[j], cu = ecu[j], cv = ecv[j];
        bool pu = rval(minr[cu], stamp) == s, pv = rval(minr[cv], stamp) == s;
        if (pu && pv) {
            int r = cu < cv ? cu : cv;
            gp[cu] = r;
            gp[cv] = r;
        } else {
            if (pu) gp[cu] = cv;
            if (pv) gp[cv] = cu;
        }
    }
}

__global__ void k_d_gjump(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                          const unsigned long long *minr, unsigned stamp, int32_t *gp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        int s = act[j];
#pragma unroll
        for (int side = 0; side < 2; side++) {
            int c = side ? ecv[j] : ecu[j];
            if (rval(minr[c], stamp) != s) continue;
            int r = gp[c];
            for (int it = 0; it < kMaxWalk; it++) {  // bounded: pointer trees
                int rr = gp[r];
                if (rr == r) break;
                r = rr;
                gp[c] = r;
            }
        }
    }
}

__global__ void k_d_tau(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                        const unsigned long long *minr, unsigned stamp, const int32_t *gp,
                        unsigned long long *tau) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        int s = act[j], cu = ecu[j], cv = ecv[j];
        if (rval(minr[cu], stamp) != s && rval(minr[cv], stamp) != s) {
            const int gu = gp[cu], gv = gp[cv];
            const unsigned long long key = rkey(stamp, s);
            if (key < tau[gu]) atomicMin(&tau[gu], key);
            if (key < tau[gv]) atomicMin(&tau[gv], key);
        }
    }
}

__global__ void k_d_accept(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                           const unsigned long long *minr, unsigned stamp, const int32_t *gp,
                           const unsigned long long *tau, int *flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= na;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j == na) {
            flag[j] = 0;
            continue;
        }
        int s = act[j], cu = ecu[j], cv = ecv[j];
        bool ptr = rval(minr[cu], stamp) == s || rval(minr[cv], stamp) == s;
        flag[j] = ptr && s < rval(tau[gp[cu]], stamp);
    }
}

// accepted edges keyed (group, rank) so a sort puts each group's chain in
// rank order; the value carries the edge's two super-vertices, the one
// whose pointer the edge is first (either for the group's mutual edge)
__global__ void k_d_emit(const int32_t *act, int64_t na, const int32_t *ecu, const int32_t *ecv,
                         const unsigned long long *minr, unsigned stamp, const int32_t *gp, const int *flag,
                         const long long *pos,
                         int sbits, unsigned long long *key, unsigned long long *val) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[j]) continue;
        const int64_t at = pos[j];
        const int s = act[j], cu = ecu[j], cv = ecv[j];
        const bool own_u = rval(minr[cu], stamp) == s;
        const unsigned Y = (unsigned)(own_u ? cu : cv), O = (unsigned)(own_u ? cv : cu);
        key[at] = ((unsigned long long)gp[cu] << sbits) | (unsigned long long)s;
        val[at] = ((unsigned long long)Y << 32) | O;
    }
}

__global__ void k_d_chain(const unsigned long long *__restrict__ key, const unsigned long long *__restrict__ val,
                          int64_t nacc, int64_t E, int sbits, const SvRec *__restrict__ sv, int2 *__restrict__ lab,
                          int32_t *__restrict__ parent, long long *__restrict__ contrib, int *__restrict__ head) {
    const unsigned long long smask = (1ull << sbits) - 1ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nacc;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[x], vv = val[x];
        const unsigned long long G = k >> sbits;
        const int s = (int)(k & smask);
        const int Y = (int)(vv >> 32), O = (int)(vv & 0xffffffffu);  // Y: the pointer's owner
        const bool h = (x == 0) || (key[x - 1] >> sbits) != G;
        int c1, c2;
        long long add;
        const SvRec ry = sv[Y];
        if (h) {
            const SvRec ro = sv[O];
            c1 = ry.root;
            c2 = ro.root;
            add = ry.size + ro.size;
        } else {
            c1 = (int)(E + (int64_t)(key[x - 1] & smask));
            c2 = ry.root;
            add = ry.size;
        }
        lab[s] = c1 < c2 ? make_int2(c1, c2) : make_int2(c2, c1);  // one sector per row
        parent[c1] = (int32_t)(E + s);
        parent[c2] = (int32_t)(E + s);
        contrib[x] = add;
        head[x] = h;
    }
}

__global__ void k_d_sizes(const unsigned long long *__restrict__ key, const unsigned long long *__restrict__ val,
                          int64_t nacc, int64_t E, int sbits, const long long *__restrict__ csum,
                          int64_t *__restrict__ lsize, int32_t *__restrict__ svpar, SvRec *__restrict__ sv) {
    const unsigned long long smask = (1ull << sbits) - 1ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nacc;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[x], vv = val[x];
        const unsigned long long G = k >> sbits;
        const int s = (int)(k & smask);
        lsize[s] = csum[x];
        svpar[(int)(vv >> 32)] = (int32_t)G;
        svpar[(int)(vv & 0xffffffffu)] = (int32_t)G;
        bool tail = (x == nacc - 1) || (key[x + 1] >> sbits) != G;
        if (tail) sv[G] = SvRec{csum[x], (int32_t)(E + s), 0};
    }
}

// the first active list: forest edges ordered by their internal end, so
// neighbouring threads touch neighbouring labels
// Rows arrive in rank order s, so the key (ru << sbits) | s sorted stably
// over the ru bits alone orders them by ru with ties in s order (no values).
__global__ void k_d_order_keys(const int32_t *ru, int64_t n, int sbits, unsigned long long *k) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        k[x] = ((unsigned long long)(unsigned)ru[x] << sbits) | (unsigned long long)x;
}
__global__ void k_d_order_act(const unsigned long long *k, int64_t n, int sbits, const int32_t *rv,
                              int32_t *act, int32_t *ecu, int32_t *ecv) {
    const unsigned long long smask = (1ull << sbits) - 1ull;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long kk = k[j];
        const int s = (int)(kk & smask);
        act[j] = s;
        ecu[j] = (int32_t)(kk >> sbits);  // ru, from the key
        ecv[j] = rv[s];
    }
}

__global__ void k_d_keep(const int32_t *__restrict__ act, int64_t na, const int *__restrict__ flag,
                         const long long *__restrict__ pos, int32_t *__restrict__ act2,
                         const int32_t *__restrict__ ecu, const int32_t *__restrict__ ecv,
                         int32_t *__restrict__ ecu2, int32_t *__restrict__ ecv2,
                         const int32_t *__restrict__ svpar) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < na;
         j += (int64_t)gridDim.x * blockDim.x) {
        int cu = ecu[j], cv = ecv[j];
        if (!flag[j]) {
            int64_t at = j - pos[j];
            act2[at] = act[j];
            ecu2[at] = svpar[cu];
            ecv2[at] = svpar[cv];
        }
    }
}

__global__ void k_d_split(const int2 *__restrict__ lab, int64_t n, int32_t *__restrict__ la,
                          int32_t *__restrict__ lb) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int2 r = lab[s];
        la[s] = r.x;
        lb[s] = r.y;
    }
}

// ------------------------------------------------ one-CTA tail of the rounds
// Once at most kTailMax forest edges are live, one CTA runs every remaining
// round: the same steps as the kernels above (bids, pointers, jumps, tau,
// acceptance, chains, sizes, keep), separated by barriers instead of
// launches, the accepted edges sorted by (group, rank) in shared memory by a
// bitonic network, and no count read on the host between rounds. The output
// orders of acceptance and keep come from shared counters: the sort orders
// the accepted edges, and the live list's order changes no result.
constexpr int kTailMax = 8192;
constexpr int kTailThreads = 1024;
constexpr size_t kTailSmem = (size_t)kTailMax * 16 + kTailMax;

__device__ __forceinline__ SegVal tail_seg(SegVal a, SegVal b) {
    SegVal r;
    r.v = b.f ? b.v : a.v + b.v;
    r.f = a.f | b.f;
    return r;
}

__global__ void __launch_bounds__(kTailThreads) k_d_tail(
    int32_t *act, int32_t *act2, int32_t *ecu, int32_t *ecu2, int32_t *ecv, int32_t *ecv2, int64_t na0, int64_t E,
    int sbits, unsigned round0, unsigned max_rounds, unsigned long long *minr, unsigned long long *tau, int32_t *gp,
    SvRec *sv, int32_t *svpar, int2 *lab, int32_t *parent, int64_t *lsize, int *status) {
    extern __shared__ unsigned long long tsm[];
    unsigned long long *skey = tsm, *sval = tsm + kTailMax;
    unsigned char *sflag = (unsigned char *)(tsm + 2 * kTailMax);
    __shared__ int s_nacc, s_nkeep;
    __shared__ SegVal s_warp[kTailThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned long long smask = (1ull << sbits) - 1ull;
    int na = (int)na0;
    unsigned round = round0;
    while (na > 0) {
        if (round - round0 >= max_rounds) {
            if (tid == 0) status[1] = 1;
            return;
        }
        const unsigned stamp = kStampTop - round;
        // bids: every live edge offers its rank to both super-vertices
        for (int j = tid; j < na; j += kTailThreads) {
            const unsigned long long key = rkey(stamp, act[j]);
            const int cu = ecu[j], cv = ecv[j];
            if (key < minr[cu]) atomicMin(&minr[cu], key);
            if (key < minr[cv]) atomicMin(&minr[cv], key);
        }
        if (tid == 0) {
            s_nacc = 0;
            s_nkeep = 0;
        }
        __syncthreads();
        // pointers (a mutual pair points both ends at its smaller label)
        for (int j = tid; j < na; j += kTailThreads) {
            const int s = act[j], cu = ecu[j], cv = ecv[j];
            const bool pu = rval(minr[cu], stamp) == s, pv = rval(minr[cv], stamp) == s;
            if (pu && pv) {
                const int r = cu < cv ? cu : cv;
                gp[cu] = r;
                gp[cv] = r;
            } else {
                if (pu) gp[cu] = cv;
                if (pv) gp[cv] = cu;
            }
        }
        __syncthreads();
        // every pointer to its tree's root
        for (int j = tid; j < na; j += kTailThreads) {
            const int s = act[j];
            for (int side = 0; side < 2; side++) {
                const int c = side ? ecv[j] : ecu[j];
                if (rval(minr[c], stamp) != s) continue;
                int r = gp[c];
                for (int it = 0; it < kMaxWalk; it++) {
                    const int rr = *(volatile int32_t *)(gp + r);
                    if (rr == r) break;
                    r = rr;
                    *(volatile int32_t *)(gp + c) = r;
                }
            }
        }
        __syncthreads();
        // tau: the smallest non-pointer edge touching each tree
        for (int j = tid; j < na; j += kTailThreads) {
            const int s = act[j], cu = ecu[j], cv = ecv[j];
            if (rval(minr[cu], stamp) != s && rval(minr[cv], stamp) != s) {
                const int gu = gp[cu], gv = gp[cv];
                const unsigned long long key = rkey(stamp, s);
                if (key < tau[gu]) atomicMin(&tau[gu], key);
                if (key < tau[gv]) atomicMin(&tau[gv], key);
            }
        }
        __syncthreads();
        // accept the pointer edges below their tree's tau; emit (group, rank)
        for (int j = tid; j < na; j += kTailThreads) {
            const int s = act[j], cu = ecu[j], cv = ecv[j];
            const bool own_u = rval(minr[cu], stamp) == s, own_v = rval(minr[cv], stamp) == s;
            const int G = gp[cu];
            const bool acc = (own_u || own_v) && s < rval(tau[G], stamp);
            sflag[j] = acc;
            if (acc) {
                const int at = atomicAdd(&s_nacc, 1);
                const unsigned Y = (unsigned)(own_u ? cu : cv), O = (unsigned)(own_u ? cv : cu);
                skey[at] = ((unsigned long long)G << sbits) | (unsigned long long)s;
                sval[at] = ((unsigned long long)Y << 32) | O;
            }
        }
        __syncthreads();
        const int nacc = s_nacc;
        if (nacc == 0) {  // every round accepts each tree's mutual edge
            if (tid == 0) status[1] = 2;
            return;
        }
        int N = 1;
        while (N < nacc) N <<= 1;
        for (int i = nacc + tid; i < N; i += kTailThreads) skey[i] = ~0ull;  // padding sorts last
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < (N >> 1); i += kTailThreads) {
                    const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long ka = skey[lo], kb = skey[hi];
                    if ((ka > kb) == up) {
                        skey[lo] = kb;
                        skey[hi] = ka;
                        const unsigned long long t = sval[lo];
                        sval[lo] = sval[hi];
                        sval[hi] = t;
                    }
                }
                __syncthreads();
            }
        }
        // chains: each thread a run of up to 8 consecutive sorted edges
        const int C = (nacc + kTailThreads - 1) / kTailThreads;  // <= kTailMax / kTailThreads
        const int x0 = tid * C;
        long long add[kTailMax / kTailThreads];
        int hd[kTailMax / kTailThreads];
#pragma unroll
        for (int q = 0; q < kTailMax / kTailThreads; q++) {
            const int x = x0 + q;
            add[q] = 0;
            hd[q] = 0;
            if (q >= C || x >= nacc) continue;
            const unsigned long long k = skey[x], vv = sval[x];
            const int s = (int)(k & smask), Y = (int)(vv >> 32), O = (int)(vv & 0xffffffffu);
            const bool h = x == 0 || (skey[x - 1] >> sbits) != (k >> sbits);
            const SvRec ry = sv[Y];
            int c1, c2;
            if (h) {
                const SvRec ro = sv[O];
                c1 = ry.root;
                c2 = ro.root;
                add[q] = ry.size + ro.size;
            } else {
                c1 = (int)(E + (int64_t)(skey[x - 1] & smask));
                c2 = ry.root;
                add[q] = ry.size;
            }
            lab[s] = c1 < c2 ? make_int2(c1, c2) : make_int2(c2, c1);
            parent[c1] = (int32_t)(E + s);
            parent[c2] = (int32_t)(E + s);
            hd[q] = h;
        }
        // sizes along each chain: a segmented inclusive sum over the runs
        SegVal agg;
        agg.v = 0;
        agg.f = 0;
#pragma unroll
        for (int q = 0; q < kTailMax / kTailThreads; q++) {
            SegVal it;
            it.v = add[q];
            it.f = hd[q];
            agg = tail_seg(agg, it);
        }
        SegVal inc = agg;
        for (int d = 1; d < 32; d <<= 1) {
            SegVal o;
            o.v = ::__shfl_up_sync(0xffffffffu, inc.v, d);
            o.f = ::__shfl_up_sync(0xffffffffu, inc.f, d);
            if (lane >= d) inc = tail_seg(o, inc);
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();  // also orders the chains' reads of sv before the writes below
        if (wid == 0) {
            SegVal w = s_warp[lane];
            for (int d = 1; d < 32; d <<= 1) {
                SegVal o;
                o.v = ::__shfl_up_sync(0xffffffffu, w.v, d);
                o.f = ::__shfl_up_sync(0xffffffffu, w.f, d);
                if (lane >= d) w = tail_seg(o, w);
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        SegVal run;
        {
            SegVal ex;
            ex.v = ::__shfl_up_sync(0xffffffffu, inc.v, 1);
            ex.f = ::__shfl_up_sync(0xffffffffu, inc.f, 1);
            if (lane == 0) {
                ex.v = 0;
                ex.f = 0;
            }
            if (wid > 0) ex = lane == 0 ? s_warp[wid - 1] : tail_seg(s_warp[wid - 1], ex);
            run = ex;
        }
#pragma unroll
        for (int q = 0; q < kTailMax / kTailThreads; q++) {
            const int x = x0 + q;
            if (q >= C || x >= nacc) continue;
            SegVal it;
            it.v = add[q];
            it.f = hd[q];
            run = tail_seg(run, it);
            const unsigned long long k = skey[x], vv = sval[x];
            const unsigned long long G = k >> sbits;
            const int s = (int)(k & smask);
            lsize[s] = run.v;
            svpar[(int)(vv >> 32)] = (int32_t)G;
            svpar[(int)(vv & 0xffffffffu)] = (int32_t)G;
            if (x == nacc - 1 || (skey[x + 1] >> sbits) != G) sv[G] = SvRec{run.v, (int32_t)(E + s), 0};
        }
        __syncthreads();
        // the edges not accepted stay live, their labels moved one hop
        for (int j = tid; j < na; j += kTailThreads) {
            if (sflag[j]) continue;
            const int at = atomicAdd(&s_nkeep, 1);
            act2[at] = act[j];
            ecu2[at] = svpar[ecu[j]];
            ecv2[at] = svpar[ecv[j]];
        }
        __syncthreads();
        na = s_nkeep;
        int32_t *t = act;
        act = act2;
        act2 = t;
        t = ecu;
        ecu = ecu2;
        ecu2 = t;
        t = ecv;
        ecv = ecv2;
        ecv2 = t;
        round++;
        __syncthreads();
    }
    if (tid == 0) status[0] = (int)(round - round0);
}

void plan_dendro(Arena &ws, const Problem &p, Dendro &o) {
    o.a = ws.take<int32_t>(p.E);
    o.b = ws.take<int32_t>(p.E);
    o.size = ws.take<int64_t>(p.E);
    o.parent = ws.take<int32_t>(2 * p.E + 1);
}

struct DScratch {
    int32_t *svpar, *gp, *act, *act2, *ecu, *ecv, *ecu2, *ecv2;
    SvRec *sv;
    int *tstat;  // one-CTA tail: [0] rounds run, [1] error
    int2 *lab;  // rows (a, b) side by side; split into the two outputs at the end
    unsigned long long *minr, *tau;  // round-stamped slots (see rkey)
    int *flag, *head;
    long long *pos, *contrib, *csum, *scan_tmp;
    SegVal *seg_tmp;
    unsigned long long *k1, *k2, *v1, *v2;
    void *radix;
};
static DScratch carve_dendro(Arena &a, const Problem &p) {
    DScratch s;
    int64_t E = p.E;
    s.svpar = a.take<int32_t>(E);
    s.sv = a.take<SvRec>(E);
    s.tstat = a.take<int>(2);
    s.lab = a.take<int2>(E);
    s.minr = a.take<unsigned long long>(E);
    s.tau = a.take<unsigned long long>(E);
    s.gp = a.take<int32_t>(E);
    s.act = a.take<int32_t>(E);
    s.act2 = a.take<int32_t>(E);
    s.ecu = a.take<int32_t>(E);
    s.ecv = a.take<int32_t>(E);
    s.ecu2 = a.take<int32_t>(E);
    s.ecv2 = a.take<int32_t>(E);
    s.flag = a.take<int>(E + 1);
    s.head = a.take<int>(E + 1);
    s.pos = a.take<long long>(E + 1);
    s.contrib = a.take<long long>(E + 1);
    s.csum = a.take<long long>(E + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(E + 1));
    s.seg_tmp = a.take<SegVal>(scan_scratch_elems(E + 1));
    s.k1 = a.take<unsigned long long>(E);
    s.k2 = a.take<unsigned long long>(E);
    s.v1 = a.take<unsigned long long>(E);
    s.v2 = a.take<unsigned long long>(E);
    s.radix = a.take<char>(radix_scratch_bytes(E));
    return s;
}
size_t dendro_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_dendro(a, p);
    return a.off;
}

dgec_status stage_dendro(Ctx *c, const Problem &p, const Csr &g, const Msf &m, Dendro &o, void *scratch) {
    cudaStream_t st = c->stream;
    int64_t E = p.E, n = m.n;
    o.rounds = 0;
    if (E == 0) return DGEC_OK;
    Arena a(scratch, SIZE_MAX);
    DScratch s = carve_dendro(a, p);
    TK(c, "k_d_init", k_d_init<<<grid_for(E + n, kBlock, kStreamCap), kBlock, 0, st>>>(
                          E, n, m.ru, m.rv, g.orig_of, s.svpar, s.sv, s.minr, s.tau,
                          o.parent, s.act, s.ecu, s.ecv));
    const int lb = p.idbits > 0 ? p.idbits : 1;
    const int sbits = bits_for((uint64_t)(n > 1 ? n - 1 : 1));
    if (n > 1) {
        const int gn = grid_for(n, kBlock, kStreamCap);
        TK(c, "k_d_order_keys", k_d_order_keys<<<gn, kBlock, 0, st>>>(m.ru, n, sbits, s.k1));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, n, sbits, sbits + lb, s.radix, &in_b));
        TK(c, "k_d_order_act", k_d_order_act<<<gn, kBlock, 0, st>>>(in_b ? s.k2 : s.k1, n, sbits, m.rv, s.act,
                                                               s.ecu, s.ecv));
    }
    int64_t na = n;
    int32_t *act = s.act, *act2 = s.act2, *ecu = s.ecu, *ecv = s.ecv, *ecu2 = s.ecu2, *ecv2 = s.ecv2;
    for (int64_t round = 0; na > 0; round++) {
        if (round >= (1 << 16))
            return set_err(c, DGEC_ERR_TIMEOUT, "dendrogram rounds exceeded %d", 1 << 16);
        if (na <= kTailMax) {  // the rest in one CTA, one launch
            CU_TRY(c, cudaFuncSetAttribute(k_d_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem));
            CU_TRY(c, cudaMemsetAsync(s.tstat, 0, 2 * sizeof(int), st));
            TK(c, "k_d_tail", k_d_tail<<<1, kTailThreads, kTailSmem, st>>>(
                                  act, act2, ecu, ecu2, ecv, ecv2, na, E, sbits, (unsigned)round,
                                  (unsigned)((1 << 16) - round), s.minr, s.tau, s.gp, s.sv, s.svpar, s.lab,
                                  o.parent, o.size, s.tstat));
            int64_t ts;
            DG_TRY(read_counters(c, (const int64_t *)s.tstat, 1, &ts));
            const int done_rounds = (int)(ts & 0xffffffff), err = (int)(ts >> 32);
            if (err == 1) return set_err(c, DGEC_ERR_TIMEOUT, "dendrogram rounds exceeded %d", 1 << 16);
            if (err) return set_err(c, DGEC_ERR_INTERNAL, "dendrogram round accepted no edge");
            o.rounds = round + done_rounds;
            break;
        }
        const int g = grid_for(na, kBlock, kStreamCap);
        const unsigned stamp = kStampTop - (unsigned)round;
        TK(c, "k_d_bid", k_d_bid<<<g, kBlock, 0, st>>>(act, na, ecu, ecv, s.minr, stamp));
        TK(c, "k_d_ptr", k_d_ptr<<<g, kBlock, 0, st>>>(act, na, ecu, ecv, s.minr, stamp, s.gp));
        TK(c, "k_d_gjump", k_d_gjump<<<g, kBlock, 0, st>>>(act, na, ecu, ecv, s.minr, stamp, s.gp));
        TK(c, "k_d_tau", k_d_tau<<<g, kBlock, 0, st>>>(act, na, ecu, ecv, s.minr, stamp, s.gp, s.tau));
        TK(c, "k_d_accept", k_d_accept<<<grid_for(na + 1, kBlock, kStreamCap), kBlock, 0, st>>>(
                                act, na, ecu, ecv, s.minr, stamp, s.gp, s.tau, s.flag));
        DG_TRY(exclusive_scan_i32(c, s.flag, s.pos, na + 1, s.scan_tmp));
        int64_t nacc;
        DG_TRY(read_counters(c, (const int64_t *)(s.pos + na), 1, &nacc));
        if (nacc <= 0) return set_err(c, DGEC_ERR_INTERNAL, "dendrogram round accepted no edge");
        TK(c, "k_d_emit", k_d_emit<<<g, kBlock, 0, st>>>(act, na, ecu, ecv, s.minr, stamp, s.gp, s.flag, s.pos, sbits,
                                                         s.k1, s.v1));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, s.v1, s.v2}, nacc, 0, lb + sbits, s.radix, &in_b));
        unsigned long long *key = in_b ? s.k2 : s.k1, *val = in_b ? s.v2 : s.v1;
        const int ga = grid_for(nacc, kBlock, kStreamCap);
        TK(c, "k_d_chain", k_d_chain<<<ga, kBlock, 0, st>>>(key, val, nacc, E, sbits, s.sv, s.lab,
                                                           o.parent, s.contrib, s.head));
        DG_TRY(segmented_inclusive_sum(c, s.contrib, s.head, s.csum, nacc, s.seg_tmp));
        TK(c, "k_d_sizes", k_d_sizes<<<ga, kBlock, 0, st>>>(key, val, nacc, E, sbits, s.csum, o.size, s.svpar,
                                                           s.sv));
        TK(c, "k_d_keep", k_d_keep<<<g, kBlock, 0, st>>>(act, na, s.flag, s.pos, act2, ecu, ecv, ecu2, ecv2,
                                                         s.svpar));
        na -= nacc;
        int32_t *t = act;
        act = act2;
        act2 = t;
        t = ecu;
        ecu = ecu2;
        ecu2 = t;
        t = ecv;
        ecv = ecv2;
        ecv2 = t;
        o.rounds = round + 1;
    }
    if (n > 0)
        TK(c, "k_d_split", k_d_split<<<grid_for(n, kBlock, kStreamCap), kBlock, 0, st>>>(s.lab, n, o.a, o.b));
    return DGEC_OK;
}

}  // namespace dgec
