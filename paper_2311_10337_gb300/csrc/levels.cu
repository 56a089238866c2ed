// Discrete dendrogram (Alg. 5, Sec. 3): components of the skeleton at
// thresholds omega_0 < ... < omega_{q-1}, and the tree D of their nesting.
//
// Alg. 5 recomputes comps(L*, omega_i) from scratch at every threshold. The
// levels are nested, so here one union-find is carried up through them: the
// skeleton edges are bucketed by the first threshold that admits them
// (w <= omega_i, the appendix's reading) and bucket i is united on top of
// the state of level i-1. Every edge is touched once in total, not q times.
//
// Union by smaller id: a hook always makes the root with the larger
// original id point to the other, so every root is the smallest member of
// its component, which is the name the outputs use. The forest itself is
// kept over internal ids (rank in (t, id) order): skeleton links join edges
// close in time, so the parent reads of one bucket stay close in memory
// instead of landing at random. A root is hooked at most once in the whole
// run, at the level where its component first meets a smaller node; that
// gives D in per-node form: merge_level[x] = that level, merge_parent[x] =
// the name of the component it joins (the root after the level's hooks).
// Only the roots hooked at a level are visited to fill merge_parent, so the
// whole build is O(|L*| + |E|), independent of q. Writing a dense label
// array per level (optional) costs one pass over the nodes per level.
//
// Condensing on D (Sec. 3, last paragraph): all merges of one level share
// the event lambda(omega_i), and equal-weight merges are condensed as one
// multi-way merge, so the condensed tree of D is that of the forest whose
// rows are D's edges with weight omega_i. build_level_rows writes those
// rows in (level, node) order; stages D1/D2 then run on them unchanged.
#include "levels.cuh"

namespace dgec {

// ---------------------------------------------------------------- buckets

// key = bucket = first i with w <= omega[i] (q when w exceeds every
// threshold: never united); val = the link's two internal ids, the end with
// the smaller original id in the high word. The sort carries the pair, so a
// bucket's hooks read one contiguous run instead of gathering.
__global__ void k_lv_keys(const int64_t *w, const int32_t *ru, const int32_t *rv, const int32_t *u,
                          const int32_t *orig_of, int64_t n, const int64_t *omega, int q,
                          unsigned long long *key, unsigned long long *val) {
    __shared__ long long om[kMaxLevels];
    for (int i = threadIdx.x; i < q; i += blockDim.x) om[i] = omega[i];
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        long long x = w[j];
        int lo = 0, hi = q;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (om[mid] >= x) hi = mid;
            else lo = mid + 1;
        }
        const int a = ru[j], b = rv[j];
        const bool a_first = orig_of[a] == u[j];
        key[j] = (unsigned long long)lo;
        val[j] = ((unsigned long long)(uint32_t)(a_first ? a : b) << 32) | (uint32_t)(a_first ? b : a);
    }
}

// boff[b] = first sorted position with bucket >= b, for b in [0, q + 1].
__global__ void k_lv_bounds(const unsigned long long *key, int64_t n, int q, int64_t *boff) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int b = s < n ? (int)key[s] : q + 1;
        int prev = s > 0 ? (int)key[s - 1] : -1;
        for (int x = prev + 1; x <= b; x++) boff[x] = s;
    }
}

__global__ void k_lv_init(int64_t E, int32_t *par, int32_t *mlevel, int32_t *mparent, int q,
                          unsigned long long *tot, int64_t *snap, int *err) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x) {
        par[x] = (int32_t)x;
        mlevel[x] = -1;
        mparent[x] = -1;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i <= q; i += blockDim.x) snap[i] = 0;
        if (threadIdx.x == 0) {
            *tot = 0;
            *err = 0;
        }
    }
}

// ------------------------------------------------------------- union-find

__device__ __forceinline__ int ld_par(const int32_t *par, int x) {
    return *(const volatile int32_t *)(par + x);
}

// Root of x with path halving (internal ids). Parents only ever move to
// ancestors (original ids strictly decrease toward the root), and a
// root's own slot is changed only by the hook's compare-and-swap, so the
// plain halving stores (made on non-roots only) are benign races.
__device__ __forceinline__ int uf_root(int32_t *par, int x) {
    for (int it = 0; it < kMaxWalk; it++) {
        int p = ld_par(par, x);
        if (p == x) return x;
        int gp = ld_par(par, p);
        if (gp == p) return p;
        *(volatile int32_t *)(par + x) = gp;
        x = gp;
    }
    return -1;
}

// Unite the bucket of level l. Roots hooked here get merge_level = l (under
// their original id) and go to the level's list (one reservation per CTA);
// the CTA-uniform loop keeps every thread in the reservation.
__global__ void __launch_bounds__(kBlock) k_lv_hook(const unsigned long long *val, const int64_t *boff,
                                                    int l, const int32_t *orig_of, int32_t *par,
                                                    int32_t *mlevel, int32_t *list, unsigned long long *tot,
                                                    int *err) {
    const int64_t lo = boff[l], hi = boff[l + 1];
    for (int64_t base = lo + (int64_t)blockIdx.x * blockDim.x; base < hi;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = base + threadIdx.x;
        int hooked = -1, hooked_orig = -1;
        if (s < hi) {
            const unsigned long long pr = val[s];
            int a = (int)(pr >> 32), b = (int)(pr & 0xffffffffull);  // orig(a) < orig(b)
            // both ends still roots: the larger original id is b, no lookup needed
            if (ld_par(par, a) == a && ld_par(par, b) == b && atomicCAS(par + b, b, a) == b) {
                hooked = b;
            } else {
                for (int it = 0; it < kMaxWalk; it++) {
                    a = uf_root(par, a);
                    b = uf_root(par, b);
                    if (a < 0 || b < 0) {
                        atomicExch(err, 1);
                        break;
                    }
                    if (a == b) break;
                    const int oa = orig_of[a], ob = orig_of[b];
                    const int big = oa > ob ? a : b, small = oa > ob ? b : a;
                    const int old = atomicCAS(par + big, big, small);
                    if (old == big) {
                        hooked = big;
                        hooked_orig = oa > ob ? oa : ob;
                        break;
                    }
                    a = old;  // `big` was hooked meanwhile: continue from its new parent
                    b = small;
                }
            }
        }
        const long long slot = cta_reserve(hooked >= 0, tot);
        if (hooked >= 0) {
            mlevel[hooked_orig >= 0 ? hooked_orig : orig_of[hooked]] = l;
            list[slot] = hooked;
        }
    }
}

// merge_parent of the roots hooked at level l: their root after the level.
// snap[l] = list start of level l; the end is the running total, recorded as
// snap[l + 1] for the next level.
__global__ void k_lv_parent(const int32_t *list, int64_t *snap, const unsigned long long *tot, int l,
                            const int32_t *orig_of, int32_t *par, int32_t *mparent, int *err) {
    const int64_t lo = snap[l], hi = (int64_t)*tot;
    for (int64_t s = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < hi;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int x = list[s];
        const int r = uf_root(par, x);
        if (r < 0) {
            atomicExch(err, 2);
            continue;
        }
        mparent[orig_of[x]] = orig_of[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) snap[l + 1] = hi;
}

// Dense labels of level l, in original-id order: every node's root, with
// full compression.
__global__ void k_lv_dense(int64_t E, int l, const int32_t *rank_of, const int32_t *orig_of, int32_t *par,
                           int32_t *dense, int *err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = rank_of[e];
        const int r = uf_root(par, x);
        if (r < 0) {
            atomicExch(err, 3);
            continue;
        }
        dense[(int64_t)l * E + e] = orig_of[r];
        if (ld_par(par, x) != r) *(volatile int32_t *)(par + x) = r;
    }
}

__global__ void k_lv_counts(int64_t E, int q, const int64_t *snap, int64_t *ncomp) {
    for (int l = threadIdx.x; l < q; l += blockDim.x) ncomp[l] = E - snap[l + 1];
}

// ------------------------------------------------------------- D as rows

// key = ((merge_level + 1) << 32) | x: nodes never merged sort first.
__global__ void k_lv_row_keys(int64_t E, const int32_t *mlevel, unsigned long long *key) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < E;
         x += (int64_t)gridDim.x * blockDim.x)
        key[x] = ((unsigned long long)(mlevel[x] + 1) << 32) | (unsigned long long)x;
}

__global__ void k_lv_rows(const unsigned long long *key, int64_t first, int64_t n, const int32_t *mparent,
                          const int32_t *rank_of, const int64_t *omega, Msf m) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[first + s];
        const int x = (int)(k & 0xffffffffull);
        const int l = (int)(k >> 32) - 1;
        const int pa = mparent[x];  // < x
        m.u[s] = pa;
        m.v[s] = x;
        m.ru[s] = rank_of[pa];
        m.rv[s] = rank_of[x];
        m.w[s] = omega[l];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        m.goff[0] = 0;
        m.goff[1] = n;
    }
}

// ------------------------------------------------------------------- host

void plan_levels(Arena &ws, const Problem &p, int q, bool dense, Levels &o) {
    o.q = q;
    o.omega = ws.take<int64_t>(kMaxLevels);
    o.mlevel = ws.take<int32_t>(p.E);
    o.mparent = ws.take<int32_t>(p.E);
    o.ncomp = ws.take<int64_t>(kMaxLevels);
    o.dense = dense ? ws.take<int32_t>((size_t)q * p.E) : nullptr;
    o.rows.u = ws.take<int32_t>(p.E);
    o.rows.v = ws.take<int32_t>(p.E);
    o.rows.ru = ws.take<int32_t>(p.E);
    o.rows.rv = ws.take<int32_t>(p.E);
    o.rows.w = ws.take<int64_t>(p.E);
    o.rows.goff = ws.take<int64_t>(2);
}

struct LvScratch {
    int32_t *par, *list;
    unsigned long long *k1, *k2, *v1, *v2, *tot;
    int64_t *boff, *snap;
    int *err;
    void *radix;
};
static LvScratch carve_levels(Arena &a, const Problem &p) {
    LvScratch s;
    const int64_t n = 2 * p.E > 1 ? 2 * p.E : 1;  // skeleton rows <= 2E; nodes E
    s.par = a.take<int32_t>(p.E);
    s.list = a.take<int32_t>(p.E);
    s.k1 = a.take<unsigned long long>(n);
    s.k2 = a.take<unsigned long long>(n);
    s.v1 = a.take<unsigned long long>(n);
    s.v2 = a.take<unsigned long long>(n);
    s.tot = a.take<unsigned long long>(1);
    s.boff = a.take<int64_t>(kMaxLevels + 2);
    s.snap = a.take<int64_t>(kMaxLevels + 1);
    s.err = a.take<int>(1);
    s.radix = a.take<char>(radix_scratch_bytes(n));
    return s;
}
size_t levels_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_levels(a, p);
    return a.off;
}

dgec_status stage_levels(Ctx *c, const Problem &p, const Csr &g, const Skel &sk, const int64_t *h_omega,
                         Levels &o, void *scratch) {
    cudaStream_t st = c->stream;
    const int64_t E = p.E, n = sk.n;
    const int q = o.q;
    o.n_merges = 0;
    CU_TRY(c, cudaMemcpyAsync(o.omega, h_omega, sizeof(int64_t) * q, cudaMemcpyHostToDevice, st));
    if (E == 0) {
        CU_TRY(c, cudaMemsetAsync(o.ncomp, 0, sizeof(int64_t) * q, st));
        return DGEC_OK;
    }
    Arena a(scratch, SIZE_MAX);
    LvScratch s = carve_levels(a, p);
    const int gE = grid_for(E, kBlock, kStreamCap);
    TK(c, "k_lv_init", k_lv_init<<<gE, kBlock, 0, st>>>(E, s.par, o.mlevel, o.mparent, q, s.tot, s.snap, s.err));
    if (n > 0) {
        const int gn = grid_for(n, kBlock, kStreamCap);
        TK(c, "k_lv_keys", k_lv_keys<<<gn, kBlock, 0, st>>>(sk.w, sk.ru, sk.rv, sk.u, g.orig_of, n, o.omega, q,
                                                           s.k1, s.v1));
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, s.v1, s.v2}, n, 0, bits_for(q), s.radix, &in_b));
        const unsigned long long *key = in_b ? s.k2 : s.k1, *val = in_b ? s.v2 : s.v1;
        TK(c, "k_lv_bounds", k_lv_bounds<<<grid_for(n + 1, kBlock, kStreamCap), kBlock, 0, st>>>(key, n, q, s.boff));
        // hook kernels read their bucket bounds on the device: no host round trip per level
        const int gh = c->num_sms * 8;
        for (int l = 0; l < q; l++) {
            TK(c, "k_lv_hook", k_lv_hook<<<gh, kBlock, 0, st>>>(val, s.boff, l, g.orig_of, s.par, o.mlevel, s.list,
                                                               s.tot, s.err));
            TK(c, "k_lv_parent", k_lv_parent<<<gh, kBlock, 0, st>>>(s.list, s.snap, s.tot, l, g.orig_of, s.par,
                                                                   o.mparent, s.err));
            if (o.dense)
                TK(c, "k_lv_dense", k_lv_dense<<<gE, kBlock, 0, st>>>(E, l, g.rank_of, g.orig_of, s.par, o.dense,
                                                                     s.err));
        }
    } else if (o.dense) {
        for (int l = 0; l < q; l++)
            TK(c, "k_lv_dense", k_lv_dense<<<gE, kBlock, 0, st>>>(E, l, g.rank_of, g.orig_of, s.par, o.dense, s.err));
    }
    TK(c, "k_lv_counts", k_lv_counts<<<1, 64, 0, st>>>(E, q, s.snap, o.ncomp));
    int64_t h[2];
    static_assert(sizeof(unsigned long long) == sizeof(int64_t), "counter width");
    DG_TRY(read_counters(c, (const int64_t *)s.tot, 1, &h[0]));
    int herr = 0;
    CU_TRY(c, cudaMemcpyAsync(&herr, s.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU_TRY(c, cudaStreamSynchronize(st));
    if (herr) return set_err(c, DGEC_ERR_TIMEOUT, "union-find walk bound exceeded (code %d)", herr);
    o.n_merges = h[0];
    return DGEC_OK;
}

dgec_status build_level_rows(Ctx *c, const Problem &p, const Csr &g, Levels &o, void *scratch) {
    cudaStream_t st = c->stream;
    const int64_t E = p.E;
    o.rows.n = o.n_merges;
    if (E == 0) {
        int64_t z[2] = {0, 0};
        CU_TRY(c, cudaMemcpyAsync(o.rows.goff, z, sizeof(z), cudaMemcpyHostToDevice, st));
        CU_TRY(c, cudaStreamSynchronize(st));
        return DGEC_OK;
    }
    Arena a(scratch, SIZE_MAX);
    LvScratch s = carve_levels(a, p);
    const int gE = grid_for(E, kBlock, kStreamCap);
    TK(c, "k_lv_row_keys", k_lv_row_keys<<<gE, kBlock, 0, st>>>(E, o.mlevel, s.k1));
    bool in_b;
    DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, E, 32, 32 + bits_for(o.q), s.radix, &in_b));
    const unsigned long long *key = in_b ? s.k2 : s.k1;
    TK(c, "k_lv_rows", k_lv_rows<<<grid_for(o.rows.n > 0 ? o.rows.n : 1, kBlock, kStreamCap), kBlock, 0, st>>>(
                           key, E - o.rows.n, o.rows.n, o.mparent, g.rank_of, o.omega, o.rows));
    return DGEC_OK;
}

}  // namespace dgec
