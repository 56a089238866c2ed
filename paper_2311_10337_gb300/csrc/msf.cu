// Stage C: minimum spanning forest of the undirected skeleton (Alg. 1)
// by Borůvka rounds, then sorted by (w, u, v) as Alg. 1 orders it.
//
// The order (w, min id, max id) is strict (a pair appears once in L*), so
// the forest is unique. Each round: every live edge between two components
// bids its w into both components with atomicMin, then the edges that match
// a component's best w bid their packed (u << 32 | v); each component hooks
// along its winning edge, a mutual pair keeps the smaller label as root,
// labels are pointer-jumped to their roots, and edges inside one component
// are dropped while the survivors are compacted for the next round.
#include "stages.cuh"

namespace dgec {

constexpr unsigned long long kMax64 = 0xFFFFFFFFFFFFFFFFull;

// A forest edge as the rounds append it: original ends (u < v), internal
// ends, weight. One 24-byte record, so that the gathers by sorted index
// after the rounds touch one sector per edge.
struct FEdge {
    int32_t u, v, ru, rv;
    int64_t w;
};

// Drop edges inside one component; compact the rest; bid w. In the first
// round every node is its own component, so the label reads are skipped.
template <bool FIRST>
__device__ __forceinline__ void filter_bid(const int32_t *u, const int32_t *v, const int64_t *w,
                                           int64_t n, const int32_t *comp, int32_t *u2, int32_t *v2,
                                           int64_t *w2, unsigned long long *cnt,
                                           unsigned long long *bw) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t wb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; wb < n;
         wb += stride) {
        int64_t x = wb + lane_id();
        bool keep = false;
        int a = 0, b = 0, ca = 0, cb = 0;
        int64_t ww = 0;
        if (x < n) {
            a = u[x];
            b = v[x];
            ww = w[x];
            ca = FIRST ? a : comp[a];
            cb = FIRST ? b : comp[b];
            keep = ca != cb;
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m == 0) continue;
        int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if ((int)lane_id() == leader) base = atomicAdd(cnt, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (keep) {
            int64_t at = (int64_t)base + __popc(m & ((1u << lane_id()) - 1u));
            u2[at] = a;
            v2[at] = b;
            w2[at] = ww;
            // read first: most bids into a large component cannot win, and
            // skipping them keeps one hot slot from serialising the grid
            // (the slot only decreases, so a stale read never skips a winner)
            unsigned long long uw = (unsigned long long)ww;
            if (uw < bw[ca]) atomicMin(&bw[ca], uw);
            if (uw < bw[cb]) atomicMin(&bw[cb], uw);
        }
    }
}

__global__ void k_filter_bid(const int32_t *u, const int32_t *v, const int64_t *w, int64_t n,
                             const int32_t *comp, int32_t *u2, int32_t *v2, int64_t *w2,
                             unsigned long long *cnt, unsigned long long *bw) {
    filter_bid<false>(u, v, w, n, comp, u2, v2, w2, cnt, bw);
}
__global__ void k_bid_uv(const int32_t *u, const int32_t *v, const int64_t *w, int64_t n,
                         const int32_t *comp, const unsigned long long *bw,
                         unsigned long long *buv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int a = u[x], b = v[x];
        unsigned long long ww = (unsigned long long)w[x];
        int ca = comp[a], cb = comp[b];
        unsigned long long key = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
        if (ww == bw[ca] && key < buv[ca]) atomicMin(&buv[ca], key);
        if (ww == bw[cb] && key < buv[cb]) atomicMin(&buv[cb], key);
    }
}

// Each component root with a winning edge hooks to the other side and, once
// per forest edge, appends it to the output.
__global__ void k_hook(int64_t E, const int32_t *comp, const unsigned long long *bw,
                       const unsigned long long *buv, int32_t *par, int32_t *mu, int32_t *mv,
                       int64_t *mw, unsigned long long *n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < E;
         base += stride) {
        int64_t x = base + lane_id();
        bool emit = false;
        int a = 0, b = 0;
        unsigned long long ww = 0;
        if (x < E && comp[x] == (int32_t)x) {
            if (bw[x] == kMax64) {
                par[x] = (int32_t)x;
            } else {
                unsigned long long key = buv[x];
                a = (int)(key >> 32);
                b = (int)(key & 0xffffffffu);
                int ca = comp[a], cb = comp[b];
                int partner = ca == (int)x ? cb : ca;
                bool mutual = buv[partner] == key;
                par[x] = (mutual && (int)x < partner) ? (int32_t)x : partner;
                emit = !mutual || (int)x < partner;
                ww = bw[x];
            }
        }
        // one counter update per warp for the forest edges it appends
        unsigned m = __ballot_sync(0xffffffffu, emit);
        if (!m) continue;
        int leader = __ffs(m) - 1;
        unsigned long long at = 0;
        if ((int)lane_id() == leader) at = atomicAdd(n_out, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (emit) {
            at += __popc(m & ((1u << lane_id()) - 1u));
            mu[at] = a;
            mv[at] = b;
            mw[at] = (int64_t)ww;
        }
    }
}

// Pointer jumping: every root walks to its new root, compressing its own
// pointer as it goes (pointers only ever move toward a root).
__global__ void k_jump(int64_t E, const int32_t *comp, int32_t *par) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (comp[x] != (int32_t)x) continue;
        int r = par[x];
        for (int it = 0; it < kMaxWalk; it++) {  // bounded: pointers form a forest
            int rr = par[r];
            if (rr == r) break;
            r = rr;
            par[x] = r;
        }
    }
}

__global__ void k_relabel(int64_t E, int32_t *comp, const int32_t *par, unsigned long long *bw,
                          unsigned long long *buv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        int c = comp[x];
        comp[x] = par[c];
    }
}

__global__ void k_reset_best(int64_t E, unsigned long long *bw, unsigned long long *buv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        bw[x] = kMax64;
        buv[x] = kMax64;
    }
}

__global__ void k_iota(int64_t E, int32_t *comp) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x)
        comp[x] = (int32_t)x;
}

// ----- the pipeline's forest stage: nodes are internal ids r; each edge
// carries its original ends (u < v) for the (w, u, v) tie-break key.

// Edges carry the labels (cu, cv) of the components at their ends; the
// labels move one hop per round (par of the old root), so no per-node
// label array is swept. Live edges: (cu, cv) labels, (u, v) original ends
// (the tie-break key), w.

// Bid w into both ends (round 1: every node is a root and nothing is
// filtered yet).
__global__ void k_m_bid(const int32_t *cu, const int32_t *cv, const int64_t *w, int64_t n,
                        unsigned long long *bw) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int a = cu[x], b = cv[x];
        unsigned long long uw = (unsigned long long)w[x];
        if (uw < bw[a]) atomicMin(&bw[a], uw);
        if (uw < bw[b]) atomicMin(&bw[b], uw);
    }
}

// Items per thread between two slot reservations of the compacting
// kernels below (one atomic on the shared counter per 2,048 items).
constexpr int kRes = 8;

// Move labels one hop to the merged roots, drop edges inside one
// component, compact the rest and bid w.
__global__ void k_m_filter_bid(const int32_t *cu, const int32_t *cv, const int32_t *u, const int32_t *v,
                               const int64_t *w, int64_t n, const int32_t *par, int32_t *cu2,
                               int32_t *cv2, int32_t *u2, int32_t *v2, int64_t *w2,
                               unsigned long long *cnt, unsigned long long *bw) {
    const int64_t tile = (int64_t)blockDim.x * kRes;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {  // CTA-uniform
        int a[kRes], b[kRes];
        unsigned keep = 0;
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            const int64_t x = base + (int64_t)q * blockDim.x + threadIdx.x;
            a[q] = b[q] = 0;
            if (x < n) {
                a[q] = par[cu[x]];
                b[q] = par[cv[x]];
                if (a[q] != b[q]) keep |= 1u << q;
            }
        }
        long long at = cta_reserve_count(__popc(keep), cnt);
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            if (!((keep >> q) & 1u)) continue;
            const int64_t x = base + (int64_t)q * blockDim.x + threadIdx.x;
            const unsigned long long uw = (unsigned long long)w[x];
            cu2[at] = a[q];
            cv2[at] = b[q];
            u2[at] = u[x];
            v2[at] = v[x];
            w2[at] = (int64_t)uw;
            at++;
            if (uw < bw[a[q]]) atomicMin(&bw[a[q]], uw);
            if (uw < bw[b[q]]) atomicMin(&bw[b[q]], uw);
        }
    }
}

__global__ void k_m_bid_uv(const int32_t *cu, const int32_t *cv, const int32_t *u, const int32_t *v,
                           const int64_t *w, int64_t n, const unsigned long long *bw,
                           unsigned long long *buv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long ww = (unsigned long long)w[x];
        int a = cu[x], b = cv[x];
        bool wa = ww == bw[a], wb = ww == bw[b];
        if (!wa && !wb) continue;
        unsigned long long key = ((unsigned long long)(unsigned)u[x] << 32) | (unsigned)v[x];
        if (wa && key < buv[a]) atomicMin(&buv[a], key);
        if (wb && key < buv[b]) atomicMin(&buv[b], key);
    }
}

// The edge that won a root's bid records itself there (one writer: keys
// are unique), with the label on its other end.
__global__ void k_m_claim(const int32_t *cu, const int32_t *cv, const int32_t *u, const int32_t *v,
                          int64_t n, const unsigned long long *buv, int32_t *bp, int32_t *win) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int a = cu[x], b = cv[x];
        unsigned long long key = ((unsigned long long)(unsigned)u[x] << 32) | (unsigned)v[x];
        if (buv[a] == key) {
            bp[a] = b;
            win[a] = (int32_t)x;
        }
        if (buv[b] == key) {
            bp[b] = a;
            win[b] = (int32_t)x;
        }
    }
}

// Over the current roots: hook along the winner (a mutual pair keeps the
// smaller label), append each forest edge once. Each thread first issues
// all its loads (8 roots), then writes: the loads of one tile are in flight
// together.
__global__ void k_m_hook(const int32_t *__restrict__ roots, int64_t nr, const unsigned long long *__restrict__ bw,
                         const unsigned long long *__restrict__ buv, const int32_t *__restrict__ bp,
                         const int32_t *__restrict__ win, const int32_t *__restrict__ u,
                         const int32_t *__restrict__ v, const int64_t *__restrict__ w,
                         const int32_t *__restrict__ rank_of, int32_t *__restrict__ par, FEdge *__restrict__ fe,
                         unsigned long long *n_out) {
    const int64_t tile = (int64_t)blockDim.x * kRes;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < nr; base += (int64_t)gridDim.x * tile) {  // CTA-uniform
        int xs[kRes], ps[kRes], wx[kRes];
        unsigned live = 0, mutual = 0;
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            const int64_t ix = base + (int64_t)q * blockDim.x + threadIdx.x;
            xs[q] = ix < nr ? roots[ix] : -1;
        }
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            ps[q] = wx[q] = 0;
            if (xs[q] < 0) continue;
            if (bw[xs[q]] != kMax64) {
                live |= 1u << q;
                ps[q] = bp[xs[q]];
                wx[q] = win[xs[q]];
            }
        }
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            if (!((live >> q) & 1u)) continue;
            const int x = xs[q], p = ps[q];
            if (bp[p] == x && buv[p] == buv[x]) mutual |= 1u << q;
        }
        unsigned emit = 0;
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            if (xs[q] < 0) continue;
            const int x = xs[q];
            if (!((live >> q) & 1u)) {
                par[x] = x;
                continue;
            }
            const bool mu = (mutual >> q) & 1u;
            par[x] = (mu && x < ps[q]) ? x : ps[q];
            if (!mu || x < ps[q]) emit |= 1u << q;
        }
        long long at = cta_reserve_count(__popc(emit), n_out);
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            if (!((emit >> q) & 1u)) continue;
            const int a = u[wx[q]], b = v[wx[q]];
            FEdge f;
            f.u = a;
            f.v = b;
            f.ru = rank_of[a];
            f.rv = rank_of[b];
            f.w = w[wx[q]];
            fe[at++] = f;
        }
    }
}

// Roots walk to their new root (own pointer compressed on the way).
__global__ void k_m_jump(const int32_t *roots, int64_t nr, int32_t *par) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < nr;
         ix += (int64_t)gridDim.x * blockDim.x) {
        int x = roots[ix];
        int r = par[x];
        for (int it = 0; it < kMaxWalk; it++) {
            int rr = par[r];
            if (rr == r) break;
            r = rr;
            par[x] = r;
        }
    }
}

// Next round's roots (old roots that stayed roots); every old root's bid
// slots are cleared. Loads first, then stores (see k_m_hook).
__global__ void k_m_next_roots(const int32_t *__restrict__ roots, int64_t nr, const int32_t *__restrict__ par,
                               unsigned long long *__restrict__ bw, unsigned long long *__restrict__ buv,
                               int32_t *__restrict__ roots2, unsigned long long *cnt) {
    const int64_t tile = (int64_t)blockDim.x * kRes;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < nr; base += (int64_t)gridDim.x * tile) {  // CTA-uniform
        int xs[kRes];
        unsigned keep = 0;
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            const int64_t ix = base + (int64_t)q * blockDim.x + threadIdx.x;
            xs[q] = ix < nr ? roots[ix] : -1;
        }
#pragma unroll
        for (int q = 0; q < kRes; q++)
            if (xs[q] >= 0 && par[xs[q]] == xs[q] && bw[xs[q]] != kMax64) keep |= 1u << q;
#pragma unroll
        for (int q = 0; q < kRes; q++) {
            if (xs[q] < 0) continue;
            bw[xs[q]] = kMax64;
            buv[xs[q]] = kMax64;
        }
        long long at = cta_reserve_count(__popc(keep), cnt);
#pragma unroll
        for (int q = 0; q < kRes; q++)
            if ((keep >> q) & 1u) roots2[at++] = xs[q];
    }
}

__global__ void k_m_init(int64_t E, int32_t *par, int32_t *roots, unsigned long long *bw,
                         unsigned long long *buv) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        par[x] = (int32_t)x;
        roots[x] = (int32_t)x;
        bw[x] = kMax64;
        buv[x] = kMax64;
    }
}

__global__ void k_pack_uv_idx(const FEdge *fe, int64_t n, int idbits, unsigned long long *k,
                              unsigned long long *val) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        k[x] = ((unsigned long long)fe[x].u << idbits) | (unsigned long long)fe[x].v;
        val[x] = (unsigned long long)x;
    }
}

__global__ void k_gather_w(const FEdge *fe, const unsigned long long *idx, int64_t n,
                           unsigned long long *k, unsigned long long *val) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long i = idx[x];
        k[x] = (unsigned long long)fe[i].w;
        val[x] = i;
    }
}

// When every w fits 32 bits the w (and graph) passes sort keys only: the
// edge index rides in the low 32 bits, which the passes do not sort on, so
// the order stays that of the previous sort among equal w (LSD stability)
// and each pass moves 8 bytes an edge instead of 16.
__global__ void k_gather_w32(const FEdge *fe, const unsigned long long *idx, int64_t n, unsigned long long *k) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long i = idx[x];
        k[x] = ((unsigned long long)fe[i].w << 32) | i;
    }
}
__global__ void k_gather_graph32(const FEdge *fe, const int32_t *egraph, const unsigned long long *kin, int64_t n,
                                 unsigned long long *k) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long i = kin[x] & 0xffffffffull;
        k[x] = ((unsigned long long)egraph[fe[i].u] << 32) | i;
    }
}

// graph of each sorted forest edge, as a sort key (graph-major output)
__global__ void k_gather_graph(const FEdge *fe, const int32_t *egraph, const unsigned long long *idx,
                               int64_t n, unsigned long long *k, unsigned long long *val) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long i = idx[x];
        k[x] = (unsigned long long)egraph[fe[i].u];
        val[x] = i;
    }
}

// goff[g] = first row of graph g in the graph-major forest (binary search)
__global__ void k_graph_offsets(const int32_t *u, const int32_t *egraph, int64_t n, int G,
                                int64_t *goff) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G;
         g += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;  // first row whose graph >= g
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (egraph[u[mid]] < g) lo = mid + 1;
            else hi = mid;
        }
        goff[g] = lo;
    }
}

__global__ void k_gather_msf(const unsigned long long *idx, unsigned long long imask, int64_t n, const FEdge *fe,
                             int32_t *u, int32_t *v, int32_t *ru, int32_t *rv, int64_t *w) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const FEdge f = fe[idx[x] & imask];
        u[x] = f.u;
        v[x] = f.v;
        ru[x] = f.ru;
        rv[x] = f.rv;
        w[x] = f.w;
    }
}

void plan_msf(Arena &ws, const Problem &p, Msf &o) {
    o.goff = ws.take<int64_t>(p.G + 1);
    o.u = ws.take<int32_t>(p.E);
    o.v = ws.take<int32_t>(p.E);
    o.ru = ws.take<int32_t>(p.E);
    o.rv = ws.take<int32_t>(p.E);
    o.w = ws.take<int64_t>(p.E);
}

struct MsfScratch {
    int32_t *par, *roots, *roots2, *bp, *win;
    int32_t *cua, *cva, *ua, *va, *cub, *cvb, *ub, *vb;
    int64_t *wa, *wb;
    FEdge *fe;
    unsigned long long *bw, *buv, *cnt;
    unsigned long long *k1, *k2, *v1, *v2;
    void *radix;
};
static MsfScratch carve_msf(Arena &a, const Problem &p) {
    MsfScratch s;
    int64_t E = p.E, S = link_cap(p);
    s.par = a.take<int32_t>(E);
    s.roots = a.take<int32_t>(E);
    s.roots2 = a.take<int32_t>(E);
    s.bp = a.take<int32_t>(E);
    s.win = a.take<int32_t>(E);
    s.cua = a.take<int32_t>(S);
    s.cva = a.take<int32_t>(S);
    s.ua = a.take<int32_t>(S);
    s.va = a.take<int32_t>(S);
    s.wa = a.take<int64_t>(S);
    s.cub = a.take<int32_t>(S);
    s.cvb = a.take<int32_t>(S);
    s.ub = a.take<int32_t>(S);
    s.vb = a.take<int32_t>(S);
    s.wb = a.take<int64_t>(S);
    s.fe = a.take<FEdge>(E);
    s.bw = a.take<unsigned long long>(E);
    s.buv = a.take<unsigned long long>(E);
    s.cnt = a.take<unsigned long long>(4);
    s.k1 = a.take<unsigned long long>(E);
    s.k2 = a.take<unsigned long long>(E);
    s.v1 = a.take<unsigned long long>(E);
    s.v2 = a.take<unsigned long long>(E);
    s.radix = a.take<char>(radix_scratch_bytes(E));
    return s;
}
size_t msf_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_msf(a, p);
    return a.off;
}

dgec_status stage_msf(Ctx *c, const Problem &p, const Csr &g, const Skel &sk, Msf &o, void *scratch) {
    cudaStream_t st = c->stream;
    o.n = 0;
    int64_t E = p.E;
    CU_TRY(c, cudaMemsetAsync(o.goff, 0, sizeof(int64_t) * (p.G + 1), st));
    if (E == 0 || sk.n == 0) return DGEC_OK;
    Arena a(scratch, SIZE_MAX);
    MsfScratch s = carve_msf(a, p);
    const int gE = grid_for(E, kBlock, kStreamCap);
    TK(c, "k_m_init", k_m_init<<<gE, kBlock, 0, st>>>(E, s.par, s.roots, s.bw, s.buv));
    CU_TRY(c, cudaMemsetAsync(s.cnt, 0, 4 * sizeof(unsigned long long), st));
    // live edges: (cu, cv) component labels, (u, v) original ends, w; the
    // first round reads the skeleton itself (labels = internal ids)
    const int32_t *ccu = sk.ru, *ccv = sk.rv, *cu = sk.u, *cv = sk.v;
    const int64_t *cw = sk.w;
    int64_t n = sk.n, nr = E;
    int32_t *roots = s.roots, *roots2 = s.roots2;
    int which = 0;
    for (int round = 0;; round++) {
        if (round >= 64) return set_err(c, DGEC_ERR_TIMEOUT, "Boruvka did not finish in 64 rounds");
        if (round == 0) {
            TK(c, "k_m_bid", k_m_bid<<<grid_for(n, kBlock, kStreamCap), kBlock, 0, st>>>(ccu, ccv, cw, n, s.bw));
        } else {
            int32_t *ncu = which ? s.cub : s.cua, *ncv = which ? s.cvb : s.cva;
            int32_t *nu = which ? s.ub : s.ua, *nv = which ? s.vb : s.va;
            int64_t *nw = which ? s.wb : s.wa;
            CU_TRY(c, cudaMemsetAsync(s.cnt, 0, sizeof(unsigned long long), st));
            TK(c, "k_m_filter_bid", k_m_filter_bid<<<grid_for(n, kBlock * kRes, kStreamCap), kBlock, 0, st>>>(
                                      ccu, ccv, cu, cv, cw, n, s.par, ncu, ncv, nu, nv, nw, s.cnt, s.bw));
            int64_t h[3];
            DG_TRY(read_counters(c, (const int64_t *)s.cnt, 3, h));
            n = h[0];
            nr = h[2];
            if (n == 0) break;
            ccu = ncu;
            ccv = ncv;
            cu = nu;
            cv = nv;
            cw = nw;
            which ^= 1;
        }
        const int gn = grid_for(n, kBlock, kStreamCap), gr = grid_for(nr, kBlock, kStreamCap),
                  grk = grid_for(nr, kBlock * kRes, kStreamCap);
        TK(c, "k_m_bid_uv", k_m_bid_uv<<<gn, kBlock, 0, st>>>(ccu, ccv, cu, cv, cw, n, s.bw, s.buv));
        TK(c, "k_m_claim", k_m_claim<<<gn, kBlock, 0, st>>>(ccu, ccv, cu, cv, n, s.buv, s.bp, s.win));
        TK(c, "k_m_hook", k_m_hook<<<grk, kBlock, 0, st>>>(roots, nr, s.bw, s.buv, s.bp, s.win, cu, cv, cw,
                                                        g.rank_of, s.par, s.fe,
                                                        s.cnt + 1));
        TK(c, "k_m_jump", k_m_jump<<<gr, kBlock, 0, st>>>(roots, nr, s.par));
        CU_TRY(c, cudaMemsetAsync(s.cnt + 2, 0, sizeof(unsigned long long), st));
        TK(c, "k_m_next_roots", k_m_next_roots<<<grk, kBlock, 0, st>>>(roots, nr, s.par, s.bw, s.buv, roots2,
                                                                    s.cnt + 2));
        int32_t *tr = roots;
        roots = roots2;
        roots2 = tr;
    }
    int64_t m;
    DG_TRY(read_counters(c, (const int64_t *)(s.cnt + 1), 1, &m));
    o.n = m;
    if (m == 0) return DGEC_OK;
    // order by (w, u, v): stable radix by the packed original ends, then by w,
    // then (batches) by graph, carrying the edge index; then gather columns
    int gm = grid_for(m, kBlock, kStreamCap);
    unsigned long long *K[2] = {s.k1, s.k2}, *Vb[2] = {s.v1, s.v2};
    int cur = 0;
    bool in_b;
    TK(c, "k_pack_uv_idx", k_pack_uv_idx<<<gm, kBlock, 0, st>>>(s.fe, m, p.idbits, K[0], Vb[0]));
    DG_TRY(radix_sort(c, RadixBuffers{K[cur], K[1 - cur], Vb[cur], Vb[1 - cur]}, m, 0, 2 * p.idbits,
                      s.radix, &in_b));
    if (in_b) cur = 1 - cur;
    if (p.tbits <= 32) {
        TK(c, "k_gather_w", k_gather_w32<<<gm, kBlock, 0, st>>>(s.fe, Vb[cur], m, K[1 - cur]));
        cur = 1 - cur;
        DG_TRY(radix_sort(c, RadixBuffers{K[cur], K[1 - cur], nullptr, nullptr}, m, 32,
                          32 + (p.tbits > 0 ? p.tbits : 1), s.radix, &in_b));
        if (in_b) cur = 1 - cur;
        if (p.G > 1) {
            TK(c, "k_gather_graph", k_gather_graph32<<<gm, kBlock, 0, st>>>(s.fe, p.egraph, K[cur], m, K[1 - cur]));
            cur = 1 - cur;
            DG_TRY(radix_sort(c, RadixBuffers{K[cur], K[1 - cur], nullptr, nullptr}, m, 32,
                              32 + bits_for((uint64_t)(p.G - 1)), s.radix, &in_b));
            if (in_b) cur = 1 - cur;
        }
    } else {
    TK(c, "k_gather_w", k_gather_w<<<gm, kBlock, 0, st>>>(s.fe, Vb[cur], m, K[1 - cur], Vb[1 - cur]));
    cur = 1 - cur;
    DG_TRY(radix_sort(c, RadixBuffers{K[cur], K[1 - cur], Vb[cur], Vb[1 - cur]}, m, 0,
                      p.tbits > 0 ? p.tbits : 1, s.radix, &in_b));
    if (in_b) cur = 1 - cur;
    if (p.G > 1) {
        TK(c, "k_gather_graph", k_gather_graph<<<gm, kBlock, 0, st>>>(s.fe, p.egraph, Vb[cur], m, K[1 - cur],
                                                                     Vb[1 - cur]));
        cur = 1 - cur;
        DG_TRY(radix_sort(c, RadixBuffers{K[cur], K[1 - cur], Vb[cur], Vb[1 - cur]}, m, 0,
                          bits_for((uint64_t)(p.G - 1)), s.radix, &in_b));
        if (in_b) cur = 1 - cur;
    }
    }
    const bool low32 = p.tbits <= 32;  // the index is the sorted key's low word
    const unsigned long long *fin = low32 ? K[cur] : Vb[cur];
    TK(c, "k_gather_msf", k_gather_msf<<<gm, kBlock, 0, st>>>(fin, low32 ? 0xffffffffull : ~0ull, m, s.fe, o.u,
                                                              o.v, o.ru, o.rv, o.w));
    TK(c, "k_graph_offsets", k_graph_offsets<<<grid_for(p.G + 1), kBlock, 0, st>>>(o.u, p.egraph, m, p.G, o.goff));
    return DGEC_OK;
}

}  // namespace dgec
