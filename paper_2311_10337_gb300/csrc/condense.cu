// Stage D2: condensed tree with minimum cluster size M (Alg. 1, condensing),
// excess-of-mass selection (Alg. 1, clusters chosen by their volume in the
// dendrogram)
// and the edge-cluster labels of Alg. 4.
//
// The paper defines these steps by citation to HDBSCAN. Readings kept
// here, identical to the oracle's:
//   - merges of equal weight are one multi-way merge (only the top merge of
//     an equal-weight run is kept), so labels depend only on the weighted
//     connectivity that Thm. 3 preserves;
//   - lambda(w) = floor((2^64 - 1) / (w + 1)); a virtual root of weight
//     infinity (lambda 0) has the components as children;
//   - top-down: a kept merge X of cluster K with >= 2 children of size >= M
//     ends K and starts one cluster per such child; with exactly one such
//     child, that child continues K; every point under a smaller child
//     leaves K at lambda(X);
//   - stabilities are exact 128-bit integers; EOM keeps a cluster when its
//     stability is >= the best total of its children; the root is never
//     kept; clusters are numbered by their smallest member id.
//
// Everything is computed by data-parallel passes: pointer jumping for the
// equal-weight runs and for "which cluster does this merge belong to",
// short upward walks (< M steps) for where a point leaves, 128-bit atomics
// for stabilities, and a rake-and-compress tree contraction over the
// cluster tree for the EOM maximisation, whose per-node update
// S = max(stab, sum of children) composes along unary chains as
// x -> max(a, c + x).
#include "stages.cuh"

namespace dgec {

typedef unsigned __int128 u128;

// Node ids: leaves [0, E), merges E + s, and one virtual root per graph at
// R0 + g (R0 = E + number of merges).
struct Gview {
    int64_t E, n, R0;
    int G;
    const int32_t *egraph;  // graph of each leaf
    const int32_t *mu;      // original lower end of each merge's forest edge
    const int64_t *eoff;    // [G+1]
    const int32_t *gM;      // [G] min cluster size per graph
};

__device__ __forceinline__ int graph_of(const Gview &g, int64_t x) {
    if (g.G == 1) return 0;  // one graph: no lookup (a merge's lookup is a random read)
    return x < g.E ? g.egraph[x] : (x < g.R0 ? g.egraph[g.mu[x - g.E]] : (int)(x - g.R0));
}

__device__ __forceinline__ unsigned long long lam_node(int64_t X, const Gview &g, const int64_t *w) {
    return X >= g.R0 ? 0ull : lambda_of(w[X - g.E]);
}

__device__ __forceinline__ int64_t node_size(int64_t X, const Gview &g, const int64_t *size) {
    if (X < g.E) return 1;
    if (X < g.R0) return size[X - g.E];
    int gr = (int)(X - g.R0);
    return g.eoff[gr + 1] - g.eoff[gr];
}

__global__ void k_c_up(int64_t E, int64_t n, const int32_t *parent, const int64_t *w, int32_t *up,
                       int *isrep) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int P = parent[E + s];
        bool rep = P < 0 || w[P - E] != w[s];
        isrep[s] = rep;
        up[s] = rep ? (int32_t)s : (int32_t)(P - E);
    }
}

// One round of in-place pointer jumping over the pointers selected by
// `Sel`: ptr[x] = ptr[ptr[x]]. Pointers only move to ancestors and fixed
// points are never written, so reading a neighbour's new or old value is
// equally valid, and every distance to the fixed point at least halves per
// round. *moved is set when any pointer changed.
struct SelAll {
    __device__ bool operator()(int64_t) const { return true; }
};
struct SelBigRep {  // big kept merges (the nodes whose cluster link is set)
    Gview gv;
    const int *isrep;
    const int64_t *size;
    __device__ bool operator()(int64_t s) const {
        return isrep[s] && size[s] >= gv.gM[graph_of(gv, gv.E + s)];
    }
};
template <class Sel>
__global__ void k_c_jump(int64_t n, int64_t off, Sel sel, int32_t *ptr, unsigned long long *moved) {
    bool any = false;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (!sel(s)) continue;
        const int64_t x = off + s;
        const int p = *(volatile int32_t *)(ptr + x);
        const int pp = *(volatile int32_t *)(ptr + p);
        if (pp != p) {
            *(volatile int32_t *)(ptr + x) = pp;
            any = true;
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(moved, 1ull);
}

// One pass of start-compressing walks, in descending index order: parents
// have larger ids than their children, so ancestors tend to be resolved
// first and later walks stop after a few steps. A walk that exceeds
// kTopWalk steps stores the ancestor it reached and flags *moved.
constexpr int kTopWalk = 1 << 12;
template <class Sel>
__global__ void k_c_top(int64_t n, int64_t off, Sel sel, int32_t *ptr, unsigned long long *moved) {
    bool cut = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = n - 1 - t;
        if (!sel(s)) continue;
        const int64_t x = off + s;
        int r = ptr[x];
        int it = 0;
        for (; it < kTopWalk; it++) {
            const int rr = ptr[r];
            if (rr == r) break;
            r = rr;
            ptr[x] = r;
        }
        cut |= it == kTopWalk;
    }
    if (__syncthreads_or(cut) && threadIdx.x == 0) atomicOr(moved, 1ull);
}

// Every selected pointer to its fixed point: one walk pass, then jumping
// rounds (checked every two) only if some walk was cut short.
template <class Sel>
static dgec_status jump_to_fixed(Ctx *c, int64_t n, int64_t off, Sel sel, int32_t *ptr,
                                 unsigned long long *moved) {
    if (n <= 0) return DGEC_OK;
    const int g = grid_for(n, kBlock, kStreamCap);
    CU_TRY(c, cudaMemsetAsync(moved, 0, sizeof(unsigned long long), c->stream));
    TK(c, "k_c_top", k_c_top<Sel><<<g, kBlock, 0, c->stream>>>(n, off, sel, ptr, moved));
    int64_t m;
    DG_TRY(read_counters(c, (const int64_t *)moved, 1, &m));
    for (int it = 0; m && it < 128; it += 2) {
        CU_TRY(c, cudaMemsetAsync(moved, 0, sizeof(unsigned long long), c->stream));
        TK(c, "k_c_jump", k_c_jump<Sel><<<g, kBlock, 0, c->stream>>>(n, off, sel, ptr, moved));
        TK(c, "k_c_jump", k_c_jump<Sel><<<g, kBlock, 0, c->stream>>>(n, off, sel, ptr, moved));
        DG_TRY(read_counters(c, (const int64_t *)moved, 1, &m));
    }
    if (m) return set_err(c, DGEC_ERR_TIMEOUT, "pointer jumping did not converge");
    return DGEC_OK;
}


// Collapsed parent of every leaf and kept merge. nbs[X - E] of a kept merge
// or virtual root X sums (1 << 32) + size over its big children: the high
// word counts them, the low word totals their sizes (below 2^31, as every
// child count and size is), so the points that leave a big X's cluster at X
// number size(X) minus the low word.
__global__ void k_c_cpar(Gview gv, const int32_t *__restrict__ parent, const int32_t *__restrict__ up,
                         const int *__restrict__ isrep, const int64_t *__restrict__ size,
                         int32_t *__restrict__ cpar, unsigned long long *__restrict__ nbs) {
    const int64_t E = gv.E;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E + gv.n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (x >= E && !isrep[x - E]) continue;
        int P = parent[x];
        int64_t cp = P < 0 ? gv.R0 + graph_of(gv, x) : E + up[P - E];
        cpar[x] = (int32_t)cp;
        if (x >= E) {
            const int64_t sz = size[x - E];
            if (sz >= gv.gM[graph_of(gv, x)]) atomicAdd(&nbs[cp - E], (1ull << 32) | (unsigned long long)sz);
        }
    }
}

// link: a big kept merge continues its parent's cluster when it is the
// parent's only big child, else it starts a cluster (link to itself);
// virtual roots link to themselves.
__global__ void k_c_link(Gview gv, const int *isrep, const int64_t *size, const int32_t *cpar,
                         const unsigned long long *nbs, int32_t *link) {
    const int64_t E = gv.E, n = gv.n;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n + gv.G;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (s >= n) {
            link[E + s] = (int32_t)(E + s);
            continue;
        }
        if (!isrep[s] || size[s] < gv.gM[graph_of(gv, E + s)]) continue;
        int64_t X = cpar[E + s];
        link[E + s] = (nbs[X - E] >> 32) >= 2 ? (int32_t)(E + s) : (int32_t)X;
    }
}


// cluster records, indexed by node id
__global__ void k_c_clusters(Gview gv, const int *isrep, const int64_t *size, const int64_t *w,
                             const int32_t *cpar, const unsigned long long *nbs, const int32_t *link, int *isc,
                             unsigned long long *cbirth, unsigned long long *cdeath,
                             int32_t *cparent) {
    const int64_t E = gv.E, n = gv.n;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n + gv.G;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t X = E + s;
        bool big = s >= n || (isrep[s] && size[s] >= gv.gM[graph_of(gv, X)]);
        if (!big) continue;
        int K = link[X];
        if ((nbs[s] >> 32) >= 2) cdeath[K] = lam_node(X, gv, w);
        if (K == (int)X) {
            isc[X] = 1;
            if (X >= gv.R0) {
                cbirth[X] = 0;
                cparent[X] = -1;
            } else {
                int64_t P = cpar[X];
                cbirth[X] = lam_node(P, gv, w);
                cparent[X] = link[P];
            }
        }
    }
}

// Per node a point can land on or walk through (kept merges, virtual
// roots): its collapsed parent, its cluster when it is big (else -1), its
// lambda and, when big, the stability share of a point leaving its cluster
// there (lambda - the cluster's birth), in one 32-byte record: each step of
// a point's walk reads one sector, and the landing needs no other lookup.
struct __align__(32) NodeRec {
    int32_t cpar;
    int32_t link;
    unsigned long long lam;
    unsigned long long share;
    unsigned long long pad;
};

// The records, and the stability the points leaving at each node give its
// cluster. Every point that leaves cluster K at the big node X does so at
// lambda(X), so together they add nf(X) * (lambda(X) - birth(K)), with nf(X)
// = size(X) minus the sizes of X's big children (the points under its small
// children, which walk up to X): one exact 128-bit add per node, summed per
// warp and cluster, instead of one per point.
__global__ void k_c_nrec(Gview gv, const int *isrep, const int64_t *size, const int64_t *w,
                         const int32_t *cpar, const int32_t *link, const unsigned long long *cbirth,
                         const unsigned long long *__restrict__ nbs, NodeRec *rec, unsigned long long *st_hi,
                         unsigned long long *st_lo) {
    const int64_t E = gv.E, n = gv.n, total = n + gv.G;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < total;
         base += stride) {  // warp-uniform
        const int64_t s = base + lane_id();
        bool has = false;
        int K = 0;
        unsigned __int128 val = 0;
        if (s < total) {
            const int64_t X = E + s;
            NodeRec r;
            r.pad = 0;
            bool write = true;
            if (s >= n) {
                r.cpar = (int32_t)X;
                r.link = link[X];
                r.lam = 0ull;
                r.share = 0ull;  // a virtual root: lambda 0, birth 0
            } else if (!isrep[s]) {
                write = false;  // never a collapsed parent
            } else {
                const int64_t sz = size[s];
                const bool big = sz >= gv.gM[graph_of(gv, X)];
                r.cpar = cpar[X];
                r.link = big ? link[X] : -1;
                r.lam = lambda_of(w[s]);
                r.share = big ? r.lam - cbirth[r.link] : 0ull;
                if (big && r.share != 0ull) {
                    const int64_t nf = sz - (int64_t)(nbs[s] & 0xffffffffull);
                    if (nf > 0) {
                        has = true;
                        K = r.link;
                        val = (unsigned __int128)(unsigned long long)nf * r.share;  // below 2^95
                    }
                }
            }
            if (write) rec[s] = r;
        }
        warp_add_u96(0xffffffffu, has, K, val, st_hi, st_lo);
    }
}

// where each point leaves: the lowest kept ancestor of size >= M (its
// stability share is counted per node above)
__global__ void k_c_points(Gview gv, const int32_t *__restrict__ cpar, const NodeRec *__restrict__ rec,
                           int32_t *__restrict__ fall_cluster, uint64_t *__restrict__ fall_lambda) {
    const int64_t E = gv.E;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E;
         p += (int64_t)gridDim.x * blockDim.x) {
        NodeRec r = rec[cpar[p] - E];
        for (int it = 0; it < kMaxWalk && r.link < 0; it++) r = rec[r.cpar - E];
        fall_cluster[p] = r.link;
        fall_lambda[p] = r.lam;
    }
}

// A child cluster's points leave the parent P at P's death: P gains
// (death - birth) * (total size of its child clusters). The sizes are summed
// here per cluster index (plain adds, no returned value, so the many
// components under a virtual root do not wait on one hot address), over the
// compacted cluster list; the product is taken when the stabilities are
// gathered.
__global__ void k_c_child_size(int64_t ncl, Gview gv, const int32_t *__restrict__ clist,
                               const int32_t *__restrict__ cparent, const int32_t *__restrict__ cidx,
                               const int64_t *__restrict__ size, unsigned long long *csz) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int K = clist[c];
        if (K >= gv.R0) continue;
        atomicAdd(&csz[cidx[cparent[K]]], (unsigned long long)size[K - gv.E]);
    }
}

// compact cluster list (ascending node id) and per-cluster arrays; only
// merges and virtual roots (node ids E + i) can be clusters, so the flags
// and their prefix sums cover those alone
__global__ void k_c_compact(int64_t E, int64_t m, const int *isc, const long long *cpos, int32_t *clist,
                            int32_t *cidx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!isc[i]) continue;
        clist[cpos[i]] = (int32_t)(E + i);
        cidx[E + i] = (int32_t)cpos[i];
    }
}

struct Eom {
    int64_t ncl;
    int64_t R0;  // node ids >= R0 are virtual roots (never selected)
    const int32_t *clist, *cidx, *cparent;  // cparent by node id
    int32_t *par;                            // compact parent, -1 root
    int *pending, *done, *state;             // state: 1 done this phase
    u128 *stab, *S, *Fa, *Fc, *Fa2, *Fc2;
    unsigned long long *acc_hi, *acc_lo;
    int32_t *ucand, *nxt, *nxt2;
    const int32_t *alist;  // open clusters this phase
    int64_t nact;
    unsigned long long *flag;  // [0] changed
};

__global__ void k_e_init(Eom e, const unsigned long long *st_hi, const unsigned long long *st_lo,
                         const unsigned long long *cbirth, const unsigned long long *cdeath,
                         const unsigned long long *csz) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < e.ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        int node = e.clist[c];
        int pn = e.cparent[node];
        e.par[c] = pn < 0 ? -1 : e.cidx[pn];
        const unsigned long long kids = csz[c];
        const u128 from_kids = kids ? (u128)(cdeath[node] - cbirth[node]) * kids : (u128)0;
        e.stab[c] = (((u128)st_hi[node] << 64) | st_lo[node]) + from_kids;
        e.done[c] = 0;
        e.acc_hi[c] = 0;
        e.acc_lo[c] = 0;
        if (pn >= 0) atomicAdd(&e.pending[e.cidx[pn]], 1);
    }
}

__device__ __forceinline__ u128 acc_of(const Eom &e, int64_t c) {
    return ((u128)e.acc_hi[c] << 64) | e.acc_lo[c];
}

// unary clusters learn their one pending child; F = (stab, acc)
__global__ void k_e_unary(Eom e) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        e.state[c] = 0;
        if (e.done[c]) continue;
        int p = e.par[c];
        if (p >= 0 && e.pending[p] == 1) e.ucand[p] = (int32_t)c;
    }
}

__global__ void k_e_fninit(Eom e) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        if (!e.done[c] && e.pending[c] == 1) {
            e.nxt[c] = e.ucand[c];
            e.Fa[c] = e.stab[c];
            e.Fc[c] = acc_of(e, c);
        } else {
            e.nxt[c] = -1;
        }
    }
}

// one synchronous doubling step: F(c) <- F(c) o F(nxt c) while nxt is unary
__global__ void k_e_double(Eom e, const int32_t *nin, int32_t *nout, const u128 *ain, const u128 *cin,
                           u128 *aout, u128 *cout) {
    bool moved = false;
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        int x = nin[c];
        u128 a = ain[c], cc = cin[c];
        if (x >= 0 && nin[x] >= 0) {
            // x is unary: compose (apply x's function first)
            u128 a2 = ain[x], c2 = cin[x];
            u128 t = cc + a2;
            a = a > t ? a : t;
            cc = cc + c2;
            x = nin[x];
            moved = true;
        }
        nout[c] = x;
        aout[c] = a;
        cout[c] = cc;
    }
    if (__any_sync(0xffffffffu, moved) && lane_id() == 0) e.flag[0] = 1;
}

// rake ready clusters (all children done)
__global__ void k_e_rake(Eom e) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        if (e.done[c] || e.pending[c] != 0) continue;
        u128 acc = acc_of(e, c);
        e.S[c] = e.stab[c] > acc ? e.stab[c] : acc;
        e.state[c] = 1;
    }
}

// unary clusters whose chain bottom was just raked resolve through F
__global__ void k_e_resolve(Eom e, const int32_t *nfin, const u128 *afin, const u128 *cfin) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        if (e.done[c] || e.pending[c] != 1) continue;
        int x = nfin[c];
        if (x < 0 || e.state[x] != 1 || e.pending[x] != 0) continue;
        u128 t = cfin[c] + e.S[x];
        e.S[c] = afin[c] > t ? afin[c] : t;
        e.state[c] = 2;
    }
}

// clusters finished this phase report to a parent that is still open
__global__ void k_e_report(Eom e) {
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < e.nact;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e.alist[ix];
        if (!e.state[c]) continue;
        int p = e.par[c];
        if (p >= 0 && !e.state[p] && !e.done[p]) {
            u128 s = e.S[c];
            atomic_add_u128(&e.acc_hi[p], &e.acc_lo[p], (unsigned long long)(s >> 64),
                            (unsigned long long)s);
            atomicSub(&e.pending[p], 1);
        }
    }
}

__global__ void k_e_commit(Eom e, int32_t *alist2, unsigned long long *n_open) {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < e.nact;
         base += (int64_t)gridDim.x * blockDim.x) {  // CTA-uniform
        int64_t ix = base + threadIdx.x;
        bool open = false;
        int64_t c = 0;
        if (ix < e.nact) {
            c = e.alist[ix];
            if (e.state[c]) e.done[c] = 1;
            open = !e.done[c];
        }
        long long at = cta_reserve(open, n_open);
        if (open) alist2[at] = (int32_t)c;
    }
}

// Small cluster trees (at most kEomSmall clusters) in one CTA. Clusters are
// numbered in ascending node id, and a parent cluster starts at a merge
// above its children's, so every child comes before its parent: one
// bottom-up sweep gives S = max(stab, sum of children's S) and the
// children's sums, one top-down sweep the highest selected ancestor-or-self.
// The sweeps are sequential (one thread, shared memory); loading and storing
// are spread over the CTA. Same results as the contraction below.
constexpr int kEomSmall = 4096;
constexpr int kEomThreads = 1024;
constexpr size_t kEomSmem = (size_t)kEomSmall * (16 + 16 + 4 + 4);
__global__ void __launch_bounds__(kEomThreads) k_e_small(Eom e, int32_t *H) {
    extern __shared__ __align__(16) unsigned long long esm[];
    u128 *sst = reinterpret_cast<u128 *>(esm);       // stab
    u128 *sacc = sst + kEomSmall;                    // children's S
    int32_t *spar = reinterpret_cast<int32_t *>(sacc + kEomSmall);
    int32_t *sh = spar + kEomSmall;
    const int n = (int)e.ncl;
    for (int c = threadIdx.x; c < n; c += kEomThreads) {
        sst[c] = e.stab[c];
        sacc[c] = 0;
        spar[c] = e.par[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < n; c++) {  // children first
            const u128 a = sacc[c], st = sst[c];
            const int p = spar[c];
            if (p >= 0) sacc[p] += st > a ? st : a;
        }
        for (int c = n - 1; c >= 0; c--) {  // parents first
            const bool sel = e.clist[c] < e.R0 && sst[c] >= sacc[c];
            const int p = spar[c];
            const int hp = p >= 0 ? sh[p] : -1;
            sh[c] = hp >= 0 ? hp : (sel ? c : -1);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += kEomThreads) {
        e.acc_hi[c] = (unsigned long long)(sacc[c] >> 64);
        e.acc_lo[c] = (unsigned long long)sacc[c];
        H[c] = sh[c];
    }
}

__global__ void k_e_iota(int64_t n, int32_t *a) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        a[x] = (int32_t)x;
}

// selection: stab(K) >= sum of children's S (ties to the parent)
__global__ void k_e_childsum(Eom e) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < e.ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        e.acc_hi[c] = 0;
        e.acc_lo[c] = 0;
    }
}
__global__ void k_e_childsum2(Eom e) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < e.ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        int p = e.par[c];
        if (p < 0) continue;
        u128 s = e.S[c];
        atomic_add_u128(&e.acc_hi[p], &e.acc_lo[p], (unsigned long long)(s >> 64), (unsigned long long)s);
    }
}
__global__ void k_e_select(Eom e, int32_t *H, int32_t *J) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < e.ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        bool sel = (e.clist[c] < e.R0) && e.stab[c] >= acc_of(e, c);
        H[c] = sel ? (int32_t)c : -1;
        J[c] = e.par[c];
    }
}

// highest selected ancestor-or-self, by synchronous doubling
__global__ void k_e_hdouble(int64_t ncl, const int32_t *Hin, const int32_t *Jin, int32_t *Hout,
                            int32_t *Jout, unsigned long long *flag) {
    bool live = false;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        int j = Jin[c];
        if (j >= 0) {
            int h = Hin[j];
            Hout[c] = h >= 0 ? h : Hin[c];
            Jout[c] = Jin[j];
            live |= Jin[j] >= 0;
        } else {
            Hout[c] = Hin[c];
            Jout[c] = -1;
        }
    }
    if (__any_sync(0xffffffffu, live) && lane_id() == 0) flag[0] = 1;
}

__global__ void k_e_labels(int64_t E, const int32_t *fall_cluster, const int32_t *cidx,
                           const int32_t *H, int32_t *lab, int *minmem) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E;
         p += (int64_t)gridDim.x * blockDim.x) {
        int L = H[cidx[fall_cluster[p]]];
        lab[p] = L;
        if (L >= 0 && (int)p < minmem[L]) atomicMin(&minmem[L], (int)p);
    }
}

__global__ void k_e_final_keys(int64_t ncl, const int32_t *H, const int *minmem, int *flag) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= ncl;
         c += (int64_t)gridDim.x * blockDim.x)
        flag[c] = (c < ncl && H[c] == (int32_t)c) ? 1 : 0;
}

__global__ void k_e_final_emit(int64_t ncl, const int *flag, const long long *pos, const int *minmem,
                               unsigned long long *k, unsigned long long *v) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[c]) continue;
        k[pos[c]] = (unsigned long long)minmem[c];
        v[pos[c]] = (unsigned long long)c;
    }
}

// Final clusters sorted by smallest member (a global edge id, so graphs
// come in order); a cluster's label is its position within its graph.
__global__ void k_e_gstart(int64_t nf, const unsigned long long *key, const int32_t *egraph,
                           int64_t *gstart, int32_t *gcount) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nf;
         x += (int64_t)gridDim.x * blockDim.x) {
        int g = egraph[key[x]];
        if (x == 0 || egraph[key[x - 1]] != g) gstart[g] = x;
        if (x == nf - 1 || egraph[key[x + 1]] != g) gcount[g] = (int32_t)(x + 1);  // end, fixed below
    }
}
__global__ void k_e_gcount(int G, const int64_t *gstart, int32_t *gcount) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        if (gcount[g] > 0) gcount[g] -= (int32_t)gstart[g];
}
__global__ void k_e_rank(int64_t nf, const unsigned long long *key, const unsigned long long *v,
                         const int32_t *egraph, const int64_t *gstart, int32_t *rank) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nf;
         x += (int64_t)gridDim.x * blockDim.x)
        rank[v[x]] = (int32_t)(x - gstart[egraph[key[x]]]);
}

__global__ void k_e_relabel(int64_t E, const int32_t *rank, int32_t *lab) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E;
         p += (int64_t)gridDim.x * blockDim.x) {
        int L = lab[p];
        lab[p] = L < 0 ? -1 : rank[L];
    }
}

__global__ void k_e_out(Eom e, Gview gv, const int64_t *size, const unsigned long long *cbirth,
                        const unsigned long long *cdeath, const int32_t *H, int32_t *cl_id,
                        int32_t *cl_parent, uint64_t *cl_birth, uint64_t *cl_death, int64_t *cl_size,
                        uint64_t *cl_hi, uint64_t *cl_lo, int32_t *cl_sel) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < e.ncl;
         c += (int64_t)gridDim.x * blockDim.x) {
        int node = e.clist[c];
        cl_id[c] = node;
        cl_parent[c] = e.cparent[node];
        cl_birth[c] = cbirth[node];
        cl_death[c] = cdeath[node];
        cl_size[c] = node_size(node, gv, size);
        cl_hi[c] = (uint64_t)(e.stab[c] >> 64);
        cl_lo[c] = (uint64_t)e.stab[c];
        bool sel = (node < e.R0) && e.stab[c] >= acc_of(e, c);
        cl_sel[c] = !sel ? 0 : (H[c] == (int32_t)c ? 2 : 1);
    }
}

void plan_condensed(Arena &ws, const Problem &p, Condensed &o) {
    int64_t E = p.E;
    o.fall_cluster = ws.take<int32_t>(E);
    o.fall_lambda = ws.take<uint64_t>(E);
    const int64_t C = E + p.G;  // clusters: at most one per merge plus the virtual roots
    o.cl_id = ws.take<int32_t>(C);
    o.cl_parent = ws.take<int32_t>(C);
    o.cl_birth = ws.take<uint64_t>(C);
    o.cl_death = ws.take<uint64_t>(C);
    o.cl_stab_hi = ws.take<uint64_t>(C);
    o.cl_stab_lo = ws.take<uint64_t>(C);
    o.cl_size = ws.take<int64_t>(C);
    o.cl_selected = ws.take<int32_t>(C);
    o.labels = ws.take<int32_t>(E);
    o.gclusters = ws.take<int32_t>(p.G);
}

struct CScratch {
    int32_t *up, *cpar, *link, *cparent, *clist, *cidx, *par, *ucand, *nxt, *nxt2, *H, *J, *H2, *J2,
        *rank, *al1, *al2;
    int *isrep, *isc, *pending, *done, *state, *minmem, *flag;
    unsigned long long *cbirth, *cdeath, *st_hi, *st_lo, *acc_hi, *acc_lo, *csz, *cnt, *k1, *k2, *v1, *v2, *jflag;
    long long *cpos, *scan_tmp;
    int64_t *gstart;
    u128 *stab, *S, *Fa, *Fc, *Fa2, *Fc2;
    void *radix;
};
static CScratch carve_condense(Arena &a, const Problem &p) {
    CScratch s;
    int64_t E = p.E, N = 2 * E + p.G + 1;  // nodes: leaves, merges, virtual roots
    s.up = a.take<int32_t>(E);
    s.isrep = a.take<int>(E);
    s.cpar = a.take<int32_t>(N);
    s.link = a.take<int32_t>(N);
    s.isc = a.take<int>(N + 1);
    s.cbirth = a.take<unsigned long long>(N);
    s.cdeath = a.take<unsigned long long>(N);
    s.cparent = a.take<int32_t>(N);
    s.st_hi = a.take<unsigned long long>(N);
    s.st_lo = a.take<unsigned long long>(N);
    s.cpos = a.take<long long>(N + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(N + 1));
    s.clist = a.take<int32_t>(E + p.G + 1);
    s.cidx = a.take<int32_t>(N);
    s.par = a.take<int32_t>(E + p.G + 1);
    s.pending = a.take<int>(E + p.G + 1);
    s.done = a.take<int>(E + p.G + 1);
    s.state = a.take<int>(E + p.G + 1);
    s.ucand = a.take<int32_t>(E + p.G + 1);
    s.nxt = a.take<int32_t>(E + p.G + 1);
    s.nxt2 = a.take<int32_t>(E + p.G + 1);
    s.stab = a.take<u128>(E + p.G + 1);
    s.S = a.take<u128>(E + p.G + 1);
    s.Fa = a.take<u128>(2 * (E + p.G + 1));  // Fa and Fc adjacent: the node records span both
    s.Fc = s.Fa + (E + p.G + 1);
    s.Fa2 = a.take<u128>(E + p.G + 1);
    s.Fc2 = a.take<u128>(E + p.G + 1);
    s.acc_hi = a.take<unsigned long long>(E + p.G + 1);
    s.acc_lo = a.take<unsigned long long>(E + p.G + 1);
    s.csz = a.take<unsigned long long>(E + p.G + 1);
    s.H = a.take<int32_t>(E + p.G + 1);
    s.J = a.take<int32_t>(E + p.G + 1);
    s.H2 = a.take<int32_t>(E + p.G + 1);
    s.J2 = a.take<int32_t>(E + p.G + 1);
    s.minmem = a.take<int>(E + p.G + 1);
    s.flag = a.take<int>(E + p.G + 2);
    s.rank = a.take<int32_t>(E + p.G + 1);
    s.gstart = a.take<int64_t>(p.G + 1);
    s.al1 = a.take<int32_t>(E + p.G + 1);
    s.al2 = a.take<int32_t>(E + p.G + 1);
    s.cnt = a.take<unsigned long long>(4);
    s.jflag = a.take<unsigned long long>(1);
    s.k1 = a.take<unsigned long long>(E + p.G + 1);
    s.k2 = a.take<unsigned long long>(E + p.G + 1);
    s.v1 = a.take<unsigned long long>(E + p.G + 1);
    s.v2 = a.take<unsigned long long>(E + p.G + 1);
    s.radix = a.take<char>(radix_scratch_bytes(E + p.G + 1));
    return s;
}
size_t condense_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_condense(a, p);
    return a.off;
}

__global__ void k_fill_i32(int *p, int64_t n, int v) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        p[x] = v;
}

dgec_status stage_condense(Ctx *c, const Problem &p, const Msf &m, const Dendro &d, Condensed &o,
                           void *scratch) {
    cudaStream_t st = c->stream;
    int64_t E = p.E, n = m.n, N = E + n + p.G;
    o.n_cl = 0;
    o.n_clusters = 0;
    CU_TRY(c, cudaMemsetAsync(o.gclusters, 0, sizeof(int32_t) * p.G, st));
    if (E == 0) return DGEC_OK;
    Gview gv{E, n, E + n, p.G, p.egraph, m.u, p.eoff, p.gM};
    Arena a(scratch, SIZE_MAX);
    CScratch s = carve_condense(a, p);
    const int gN = grid_for(N, kBlock, kStreamCap), gE = grid_for(E, kBlock, kStreamCap),
              gn = grid_for(n + p.G, kBlock, kStreamCap);
    // big-child counts and sizes of node ids E .. N: in cpos, unused until the cluster scan
    unsigned long long *nbs = reinterpret_cast<unsigned long long *>(s.cpos);
    CU_TRY(c, cudaMemsetAsync(nbs, 0, sizeof(unsigned long long) * (n + p.G), st));
    CU_TRY(c, cudaMemsetAsync(s.isc + E, 0, sizeof(int) * (n + p.G + 1), st));
    CU_TRY(c, cudaMemsetAsync(s.cdeath, 0, sizeof(unsigned long long) * N, st));
    CU_TRY(c, cudaMemsetAsync(s.st_hi, 0, sizeof(unsigned long long) * N, st));
    CU_TRY(c, cudaMemsetAsync(s.st_lo, 0, sizeof(unsigned long long) * N, st));
    if (n > 0) {
        TK(c, "k_c_up", k_c_up<<<gn, kBlock, 0, st>>>(E, n, d.parent, m.w, s.up, s.isrep));
        DG_TRY(jump_to_fixed(c, n, 0, SelAll{}, s.up, s.jflag));
    }
    TK(c, "k_c_cpar", k_c_cpar<<<gN, kBlock, 0, st>>>(gv, d.parent, s.up, s.isrep, d.size, s.cpar, nbs));
    TK(c, "k_c_link", k_c_link<<<gn, kBlock, 0, st>>>(gv, s.isrep, d.size, s.cpar, nbs, s.link));
    DG_TRY(jump_to_fixed(c, n, E, SelBigRep{gv, s.isrep, d.size}, s.link, s.jflag));
    TK(c, "k_c_clusters", k_c_clusters<<<gn, kBlock, 0, st>>>(gv, s.isrep, d.size, m.w, s.cpar, nbs, s.link,
                                                             s.isc, s.cbirth, s.cdeath, s.cparent));
    // the node records live in the EOM phase's Fa and Fc arrays (adjacent, not in use yet)
    NodeRec *nrec = reinterpret_cast<NodeRec *>(s.Fa);
    TK(c, "k_c_nrec", k_c_nrec<<<gn, kBlock, 0, st>>>(gv, s.isrep, d.size, m.w, s.cpar, s.link, s.cbirth, nbs,
                                                     nrec, s.st_hi, s.st_lo));
    TK(c, "k_c_points", k_c_points<<<gE, kBlock, 0, st>>>(gv, s.cpar, nrec, o.fall_cluster, o.fall_lambda));
    // cluster flags of node ids E .. N (the last one a zero sentinel)
    DG_TRY(exclusive_scan_i32(c, s.isc + E, s.cpos, n + p.G + 1, s.scan_tmp));
    int64_t ncl;
    DG_TRY(read_counters(c, (const int64_t *)(s.cpos + n + p.G), 1, &ncl));
    TK(c, "k_c_compact", k_c_compact<<<gn, kBlock, 0, st>>>(E, n + p.G, s.isc + E, s.cpos, s.clist, s.cidx));
    o.n_cl = ncl;
    CU_TRY(c, cudaMemsetAsync(s.csz, 0, sizeof(unsigned long long) * (ncl + 1), st));
    TK(c, "k_c_child_size", k_c_child_size<<<grid_for(ncl, kBlock, kStreamCap), kBlock, 0, st>>>(
                                ncl, gv, s.clist, s.cparent, s.cidx, d.size, s.csz));
    // ---- excess of mass over the cluster tree
    Eom e;
    e.ncl = ncl;
    e.R0 = E + n;
    e.clist = s.clist;
    e.cidx = s.cidx;
    e.cparent = s.cparent;
    e.par = s.par;
    e.pending = s.pending;
    e.done = s.done;
    e.state = s.state;
    e.stab = s.stab;
    e.S = s.S;
    e.Fa = s.Fa;
    e.Fc = s.Fc;
    e.Fa2 = s.Fa2;
    e.Fc2 = s.Fc2;
    e.acc_hi = s.acc_hi;
    e.acc_lo = s.acc_lo;
    e.ucand = s.ucand;
    e.nxt = s.nxt;
    e.nxt2 = s.nxt2;
    const int gc = grid_for(ncl + 1, kBlock, kStreamCap);
    e.flag = s.cnt + 2;
    CU_TRY(c, cudaMemsetAsync(s.pending, 0, sizeof(int) * (ncl + 1), st));
    TK(c, "k_e_init", k_e_init<<<gc, kBlock, 0, st>>>(e, s.st_hi, s.st_lo, s.cbirth, s.cdeath, s.csz));
    int32_t *Hi = s.H;  // highest selected ancestor-or-self of every cluster
    if (ncl <= kEomSmall) {
        CU_TRY(c, cudaFuncSetAttribute(k_e_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEomSmem));
        TK(c, "k_e_small", k_e_small<<<1, kEomThreads, kEomSmem, st>>>(e, Hi));
    } else {
    TK(c, "k_e_iota", k_e_iota<<<gc, kBlock, 0, st>>>(ncl, s.al1));
    int32_t *al = s.al1, *al2 = s.al2;
    int64_t nact = ncl;
    const int kMaxDouble = 40;  // chains are shorter than 2^31
    for (int phase = 0;; phase++) {
        if (phase > 4096) return set_err(c, DGEC_ERR_TIMEOUT, "EOM contraction exceeded 4096 phases");
        e.alist = al;
        e.nact = nact;
        const int ga = grid_for(nact, kBlock, kStreamCap);
        TK(c, "k_e_unary", k_e_unary<<<ga, kBlock, 0, st>>>(e));
        TK(c, "k_e_fninit", k_e_fninit<<<ga, kBlock, 0, st>>>(e));
        int32_t *ni = s.nxt, *no = s.nxt2;
        u128 *ai = s.Fa, *ao = s.Fa2, *ci = s.Fc, *co = s.Fc2;
        // synchronous doubling until no pointer moves (checked every 2 steps)
        for (int it = 0; it < kMaxDouble; it++) {
            if ((it & 1) == 0) CU_TRY(c, cudaMemsetAsync(e.flag, 0, sizeof(unsigned long long), st));
            TK(c, "k_e_double", k_e_double<<<ga, kBlock, 0, st>>>(e, ni, no, ai, ci, ao, co));
            int32_t *t = ni;
            ni = no;
            no = t;
            u128 *ta = ai;
            ai = ao;
            ao = ta;
            ta = ci;
            ci = co;
            co = ta;
            if (it & 1) {
                int64_t moved;
                DG_TRY(read_counters(c, (const int64_t *)e.flag, 1, &moved));
                if (!moved) break;
            }
        }
        TK(c, "k_e_rake", k_e_rake<<<ga, kBlock, 0, st>>>(e));
        TK(c, "k_e_resolve", k_e_resolve<<<ga, kBlock, 0, st>>>(e, ni, ai, ci));
        TK(c, "k_e_report", k_e_report<<<ga, kBlock, 0, st>>>(e));
        CU_TRY(c, cudaMemsetAsync(s.cnt, 0, sizeof(unsigned long long), st));
        TK(c, "k_e_commit", k_e_commit<<<ga, kBlock, 0, st>>>(e, al2, s.cnt));
        int64_t open;
        DG_TRY(read_counters(c, (const int64_t *)s.cnt, 1, &open));
        if (open == 0) break;
        int32_t *t = al;
        al = al2;
        al2 = t;
        nact = open;
    }
    TK(c, "k_e_childsum", k_e_childsum<<<gc, kBlock, 0, st>>>(e));
    TK(c, "k_e_childsum2", k_e_childsum2<<<gc, kBlock, 0, st>>>(e));
    TK(c, "k_e_select", k_e_select<<<gc, kBlock, 0, st>>>(e, s.H, s.J));
    int32_t *Ji = s.J, *Ho = s.H2, *Jo = s.J2;
    for (int it = 0; it < kMaxDouble; it++) {
        if ((it & 1) == 0) CU_TRY(c, cudaMemsetAsync(e.flag, 0, sizeof(unsigned long long), st));
        TK(c, "k_e_hdouble", k_e_hdouble<<<gc, kBlock, 0, st>>>(ncl, Hi, Ji, Ho, Jo, e.flag));
        int32_t *t = Hi;
        Hi = Ho;
        Ho = t;
        t = Ji;
        Ji = Jo;
        Jo = t;
        if (it & 1) {
            int64_t live;
            DG_TRY(read_counters(c, (const int64_t *)e.flag, 1, &live));
            if (!live) break;
        }
    }
    }
    TK(c, "k_fill_i32", k_fill_i32<<<gc, kBlock, 0, st>>>(s.minmem, ncl + 1, INT_MAX));
    TK(c, "k_e_labels", k_e_labels<<<gE, kBlock, 0, st>>>(E, o.fall_cluster, s.cidx, Hi, o.labels, s.minmem));
    TK(c, "k_e_final_keys", k_e_final_keys<<<gc, kBlock, 0, st>>>(ncl, Hi, s.minmem, s.flag));
    DG_TRY(exclusive_scan_i32(c, s.flag, s.cpos, ncl + 1, s.scan_tmp));
    int64_t nf;
    DG_TRY(read_counters(c, (const int64_t *)(s.cpos + ncl), 1, &nf));
    o.n_clusters = (int32_t)nf;
    if (nf > 0) {
        TK(c, "k_e_final_emit", k_e_final_emit<<<gc, kBlock, 0, st>>>(ncl, s.flag, s.cpos, s.minmem, s.k1, s.v1));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, s.v1, s.v2}, nf, 0, p.idbits > 0 ? p.idbits : 1,
                          s.radix, &in_b));
        unsigned long long *kk = in_b ? s.k2 : s.k1, *vv = in_b ? s.v2 : s.v1;
        const int gf = grid_for(nf, kBlock, kStreamCap);
        TK(c, "k_e_gstart", k_e_gstart<<<gf, kBlock, 0, st>>>(nf, kk, p.egraph, s.gstart, o.gclusters));
        TK(c, "k_e_gcount", k_e_gcount<<<grid_for(p.G), kBlock, 0, st>>>(p.G, s.gstart, o.gclusters));
        TK(c, "k_e_rank", k_e_rank<<<gf, kBlock, 0, st>>>(nf, kk, vv, p.egraph, s.gstart, s.rank));
        TK(c, "k_e_relabel", k_e_relabel<<<gE, kBlock, 0, st>>>(E, s.rank, o.labels));
    }
    TK(c, "k_e_out", k_e_out<<<gc, kBlock, 0, st>>>(e, gv, d.size, s.cbirth, s.cdeath, Hi, o.cl_id, o.cl_parent,
                                   o.cl_birth, o.cl_death, o.cl_size, o.cl_stab_hi, o.cl_stab_lo,
                                   o.cl_selected));
    return DGEC_OK;
}

}  // namespace dgec
