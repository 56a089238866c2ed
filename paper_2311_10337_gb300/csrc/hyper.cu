// Dynamic hypergraphs (Sec. 4.4): hyperedges e = (S_e, t_e) are the nodes of
// the line graph; two hyperedges sharing a vertex are joined with weight
// |t_r - t_s|. At a vertex the incident hyperedges form a clique whose
// local MST (ties by id) is the path through them in (t, id) order
// (undirected), or, for directed hyperedges with sources S_e and targets
// R_e, what Alg. 2 gives on the vertex's in-list (hyperedges with the
// vertex as a target) and out-list (as a source). The skeleton is the union
// of the local MSTs as a set; Alg. 1 then runs on it through the forest,
// dendrogram and condense stages of the graph path.
//
// Lists: every hyperedge gets its internal id r = rank in (t, id) order
// (one radix sort over the time bits, as for graph edges); memberships are
// scattered into per-vertex segments and each segment is sorted by r, so a
// list is in (t, id) order. Each slot also keeps its vertex (written by the
// scatter; a segment sort only permutes within one vertex).
//
// Links: one per membership at most (undirected: slot x links to slot x-1
// of the same vertex; directed: every in-slot emits Alg. 2's type-1 link
// and every out-slot its type-2 link, as rank arithmetic on the two sorted
// lists). A pair that shares several vertices can be emitted at each, so
// the links are keyed (min r, max r), sorted once and kept once.
#include <algorithm>

#include "hyper.cuh"

namespace dgec {

// flags: [0] bad offsets, [1] vertex out of range, [2] t min, [3] t max,
// [4] vertex repeated in a member set, [5] vertex both source and target
constexpr int kHFlags = 8;

__global__ void k_h_init_flags(long long *f) {
    for (int i = 0; i < kHFlags; i++) f[i] = 0;
    f[2] = LLONG_MAX;
    f[3] = LLONG_MIN;
}

// off[0] == 0, off non-decreasing, off[E] == M
__global__ void k_h_check_off(const int64_t *off, int64_t E, int64_t M, long long *f) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= E;
         e += (int64_t)gridDim.x * blockDim.x) {
        bool bad = (e == 0 && off[0] != 0) || (e == E && off[E] != M) || (e < E && off[e + 1] < off[e]);
        if (bad) atomicAdd((unsigned long long *)&f[0], 1ull);
    }
}

__global__ void k_h_count(const int32_t *vert, int64_t M, int64_t V, int *deg, long long *f) {
    // warp-strided loop so warp_agg_inc sees whole warps
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = stride >> 5;
    for (int64_t wb = warp_global * 32; wb < M; wb += nwarps * 32) {
        const int64_t m = wb + lane_id();
        const bool in = m < M;
        const int v = in ? vert[m] : 0;
        const bool ok = in && v >= 0 && v < V;
        if (in && !ok) atomicAdd((unsigned long long *)&f[1], 1ull);
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) warp_agg_inc(deg, v, act);
    }
}

__global__ void k_h_tminmax(const int64_t *t, int64_t E, long long *f) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, (long long)t[e]);
        hi = max(hi, (long long)t[e]);
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if (lane_id() == 0) {
        atomicMin(&f[2], lo);
        atomicMax(&f[3], hi);
    }
}

__global__ void k_h_pack(const int64_t *t, int64_t E, long long tmin, int idbits, unsigned long long *k) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        k[e] = ((unsigned long long)(t[e] - tmin) << idbits) | (unsigned long long)e;
}

__global__ void k_h_rank_init(const unsigned long long *ks, int64_t E, long long tmin, int idbits,
                              int32_t *orig_of, int32_t *rank_of, int64_t *it) {
    const unsigned long long mask = (1ull << idbits) - 1ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
         r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ks[r];
        const int32_t e = (int32_t)(k & mask);
        orig_of[r] = e;
        rank_of[e] = (int32_t)r;
        it[r] = (int64_t)(k >> idbits) + tmin;
    }
}

// Membership m of hyperedge e (off[e] <= m < off[e+1]) goes to its
// vertex's segment as key r = rank_of[e]; the slot remembers the vertex.
__global__ void k_h_scatter(const int64_t *off, int64_t E, const int32_t *vert, int64_t M,
                            const int32_t *rank_of, const int64_t *voff, int *cur,
                            unsigned long long *keys, int32_t *vx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = stride >> 5;
    for (int64_t wb = warp_global * 32; wb < M; wb += nwarps * 32) {
        const int64_t m = wb + lane_id();
        const bool ok = m < M;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (!ok) continue;
        int64_t lo = 0, hi = E + 1;  // first index with off[idx] > m
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= m) lo = mid + 1;
            else hi = mid;
        }
        const int64_t e = lo - 1;
        const int v = vert[m];
        const int slot = warp_agg_inc(cur, v, act);
        keys[voff[v] + slot] = (unsigned long long)rank_of[e];
        vx[voff[v] + slot] = v;
    }
}

__global__ void k_h_unpack(const unsigned long long *keys, int64_t M, const int32_t *orig_of, const int64_t *it,
                           HyperLists L, long long *f) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)keys[x];
        L.r[x] = r;
        L.id[x] = orig_of[r];
        L.tt[x] = it[r];
        if (x > 0 && L.vx[x - 1] == L.vx[x] && (int32_t)keys[x - 1] == r)
            atomicAdd((unsigned long long *)&f[4], 1ull);
    }
}

__device__ __forceinline__ unsigned long long pair_key(int a, int b, int idbits) {
    const unsigned long long lo = (unsigned)(a < b ? a : b), hi = (unsigned)(a < b ? b : a);
    return (lo << idbits) | hi;
}

// undirected: the path through each vertex's list
__global__ void k_h_path(HyperLists L, int64_t M, int idbits, unsigned long long *lk) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = ~0ull;
        if (x > 0 && L.vx[x - 1] == L.vx[x] && L.r[x - 1] != L.r[x]) k = pair_key(L.r[x - 1], L.r[x], idbits);
        lk[x] = k;
    }
}

__device__ __forceinline__ int64_t h_lower(const int64_t *a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t h_upper(const int64_t *a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// directed, type 1: in-slot p at vertex i links to the first out-slot q of
// i with t_q >= t_p (in before out at equal t): index #{q : t_q < t_p}.
__global__ void k_h_type1(HyperLists in, int64_t Md, HyperLists out, int idbits, unsigned long long *lk) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < Md;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int i = in.vx[x];
        const int64_t ob = out.voff[i], nout = out.voff[i + 1] - ob;
        const int64_t a = h_lower(out.tt + ob, nout, in.tt[x]);
        unsigned long long k = ~0ull;
        if (a < nout && out.r[ob + a] != in.r[x]) k = pair_key(in.r[x], out.r[ob + a], idbits);
        lk[x] = k;
    }
}

// directed, type 2: out-slot q_m (m >= 1) at vertex i links to the in-slot
// p_{b-1}, b = #{p : t_p <= t(q_{m-1})}, when b >= 1. Also rejects a
// hyperedge that has i both as a source and as a target.
__global__ void k_h_type2(HyperLists in, HyperLists out, int64_t Ms, int64_t Md, int idbits,
                          unsigned long long *lk, long long *f) {
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < Ms;
         y += (int64_t)gridDim.x * blockDim.x) {
        const int i = out.vx[y];
        const int q = out.r[y];
        const int64_t ib = in.voff[i], nin = in.voff[i + 1] - ib;
        {  // in-list sorted by r: exact membership test
            int64_t lo = 0, hi = nin;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (in.r[ib + mid] < q) lo = mid + 1;
                else hi = mid;
            }
            if (lo < nin && in.r[ib + lo] == q) atomicAdd((unsigned long long *)&f[5], 1ull);
        }
        unsigned long long k = ~0ull;
        if (y > out.voff[i]) {
            const int64_t b = h_upper(in.tt + ib, nin, out.tt[y - 1]);
            if (b >= 1 && in.r[ib + b - 1] != q) k = pair_key(in.r[ib + b - 1], q, idbits);
        }
        lk[Md + y] = k;
    }
}

__global__ void k_h_uflag(const unsigned long long *lk, int64_t L, int *flag) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= L;
         x += (int64_t)gridDim.x * blockDim.x)
        flag[x] = x < L && lk[x] != ~0ull && (x == 0 || lk[x] != lk[x - 1]);
}

__global__ void k_h_links(const unsigned long long *lk, int64_t L, const int *flag, const long long *pos,
                          int idbits, const int32_t *orig_of, const int64_t *it, Skel sk) {
    const unsigned long long mask = (1ull << idbits) - 1ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[x]) continue;
        const int a = (int)(lk[x] >> idbits), b = (int)(lk[x] & mask);  // a < b: t_a <= t_b
        const int64_t at = pos[x];
        const int ua = orig_of[a], ub = orig_of[b];
        sk.ru[at] = a;
        sk.rv[at] = b;
        sk.u[at] = ua < ub ? ua : ub;
        sk.v[at] = ua < ub ? ub : ua;
        sk.w[at] = it[b] - it[a];
    }
}

// ------------------------------------------------------------------- host

void plan_hyper(Arena &ws, const HyperProblem &h, Csr &g, HyperLists &S, HyperLists &D, Skel &sk) {
    memset(&g, 0, sizeof(g));
    g.orig_of = ws.take<int32_t>(h.E);
    g.rank_of = ws.take<int32_t>(h.E);
    g.it = ws.take<int64_t>(h.E);
    auto lists = [&](HyperLists &L, int64_t M) {
        L.voff = ws.take<int64_t>(h.V + 1);
        L.id = ws.take<int32_t>(M);
        L.r = ws.take<int32_t>(M);
        L.tt = ws.take<int64_t>(M);
        L.vx = ws.take<int32_t>(M);
    };
    lists(S, h.Ms);
    if (h.directed) lists(D, h.Md);
    else memset(&D, 0, sizeof(D));
    const int64_t L = h.Ms + h.Md;
    sk.u = ws.take<int32_t>(L);
    sk.v = ws.take<int32_t>(L);
    sk.ru = ws.take<int32_t>(L);
    sk.rv = ws.take<int32_t>(L);
    sk.w = ws.take<int64_t>(L);
    sk.knn = nullptr;
    sk.core = nullptr;
    sk.n = 0;
}

struct HScratch {
    long long *f, *scan_tmp, *pos;
    int *deg_s, *deg_d, *flag;
    unsigned long long *k1, *k2;
    SegSort seg;
    void *radix;
};
static HScratch carve_hyper(Arena &a, const HyperProblem &h) {
    HScratch s;
    const int64_t L = h.Ms + h.Md, n = std::max<int64_t>(std::max<int64_t>(h.E, L), 1);
    s.f = a.take<long long>(kHFlags);
    s.deg_s = a.take<int>(h.V + 1);
    s.deg_d = a.take<int>(h.V + 1);
    s.flag = a.take<int>(L + 1);
    s.pos = a.take<long long>(L + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(std::max<int64_t>(L + 1, h.V + 1)));
    s.k1 = a.take<unsigned long long>(n);
    s.k2 = a.take<unsigned long long>(n);
    carve_segsort(a, h.V, std::max<int64_t>(std::max<int64_t>(h.Ms, h.Md), 1), s.seg);
    s.radix = a.take<char>(radix_scratch_bytes(n));
    return s;
}
size_t hyper_scratch_bytes(const HyperProblem &h) {
    Arena a(nullptr, 0);
    carve_hyper(a, h);
    return a.off;
}

__global__ void k_h_set(long long *p, long long v) { *p = v; }

static dgec_status build_lists(Ctx *c, const HyperProblem &h, const int64_t *off, const int32_t *vert, int64_t M,
                               int *deg, const Csr &g, int idbits, HyperLists &L, HScratch &s) {
    cudaStream_t st = c->stream;
    const int64_t V = h.V;
    if (V > 0) DG_TRY(exclusive_scan_i32(c, deg, (long long *)L.voff, V, s.scan_tmp));
    TK(c, "k_h_set", k_h_set<<<1, 1, 0, st>>>((long long *)L.voff + V, M));
    if (M == 0) return DGEC_OK;
    CU_TRY(c, cudaMemsetAsync(deg, 0, sizeof(int) * (V + 1), st));
    TK(c, "k_h_scatter", k_h_scatter<<<grid_for(M, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                             off, h.E, vert, M, g.rank_of, L.voff, deg, s.k1, L.vx));
    DG_TRY(sort_segments(c, V, s.k1, L.voff, s.seg, idbits));
    TK(c, "k_h_unpack", k_h_unpack<<<grid_for(M, kBlock, kStreamCap), kBlock, 0, st>>>(s.k1, M, g.orig_of, g.it, L, s.f));
    return DGEC_OK;
}

dgec_status stage_hyper(Ctx *c, Problem &p, const HyperProblem &h, Csr &g, HyperLists &S, HyperLists &D, Skel &sk,
                        void *scratch) {
    cudaStream_t st = c->stream;
    Arena a(scratch, SIZE_MAX);
    HScratch s = carve_hyper(a, h);
    const int64_t E = h.E, V = h.V;
    sk.n = 0;
    TK(c, "k_h_init_flags", k_h_init_flags<<<1, 1, 0, st>>>(s.f));
    CU_TRY(c, cudaMemsetAsync(s.deg_s, 0, sizeof(int) * (V + 1), st));
    CU_TRY(c, cudaMemsetAsync(s.deg_d, 0, sizeof(int) * (V + 1), st));
    TK(c, "k_h_check_off", k_h_check_off<<<grid_for(E + 1, kBlock, kStreamCap), kBlock, 0, st>>>(h.s_off, E, h.Ms, s.f));
    if (h.directed)
        TK(c, "k_h_check_off", k_h_check_off<<<grid_for(E + 1, kBlock, kStreamCap), kBlock, 0, st>>>(h.d_off, E, h.Md, s.f));
    if (h.Ms > 0)
        TK(c, "k_h_count", k_h_count<<<grid_for(h.Ms, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                               h.s_vert, h.Ms, V, s.deg_s, s.f));
    if (h.directed && h.Md > 0)
        TK(c, "k_h_count", k_h_count<<<grid_for(h.Md, kBlock, (int64_t)c->num_sms * 16), kBlock, 0, st>>>(
                               h.d_vert, h.Md, V, s.deg_d, s.f));
    if (E > 0) TK(c, "k_h_tminmax", k_h_tminmax<<<grid_for(E, kBlock, 1024), kBlock, 0, st>>>(h.t, E, s.f));
    int64_t f[kHFlags];
    DG_TRY(read_counters(c, (const int64_t *)s.f, kHFlags, f));
    if (f[0]) return set_err(c, DGEC_ERR_INVALID_ARG, "member offsets must start at 0, not decrease, end at the member count");
    if (f[1]) return set_err(c, DGEC_ERR_VERTEX_RANGE, "%lld members outside [0, n_vertices)", (long long)f[1]);
    p.tmin = E > 0 ? f[2] : 0;
    const uint64_t span = E > 0 ? (uint64_t)(f[3] - f[2]) : 0;
    p.idbits = bits_for((uint64_t)(E > 1 ? E - 1 : 1));
    p.tbits = bits_for(span);
    if (p.idbits + p.tbits > 64 || 2 * p.idbits > 64)
        return set_err(c, DGEC_ERR_TOO_LARGE, "time span %llu needs %d bits + %d id bits > 64",
                       (unsigned long long)span, p.tbits, p.idbits);
    if (E == 0) {  // no members either (offsets checked): empty lists
        CU_TRY(c, cudaMemsetAsync(S.voff, 0, sizeof(int64_t) * (V + 1), st));
        if (h.directed) CU_TRY(c, cudaMemsetAsync(D.voff, 0, sizeof(int64_t) * (V + 1), st));
        return DGEC_OK;
    }
    // hyperedges in (t, id) order: internal ids
    const int gE = grid_for(E, kBlock, kStreamCap);
    TK(c, "k_h_pack", k_h_pack<<<gE, kBlock, 0, st>>>(h.t, E, p.tmin, p.idbits, s.k1));
    {
        bool in_b;
        DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, E, p.idbits, p.idbits + p.tbits, s.radix,
                          &in_b));
        TK(c, "k_h_rank_init", k_h_rank_init<<<gE, kBlock, 0, st>>>(in_b ? s.k2 : s.k1, E, p.tmin, p.idbits,
                                                                   g.orig_of, g.rank_of, g.it));
    }
    DG_TRY(build_lists(c, h, h.s_off, h.s_vert, h.Ms, s.deg_s, g, p.idbits, S, s));
    if (h.directed) DG_TRY(build_lists(c, h, h.d_off, h.d_vert, h.Md, s.deg_d, g, p.idbits, D, s));
    // links, keyed (min r, max r)
    const int64_t L = h.directed ? h.Ms + h.Md : h.Ms;
    if (L == 0) {
        DG_TRY(read_counters(c, (const int64_t *)s.f, kHFlags, f));
        if (f[4]) return set_err(c, DGEC_ERR_SELF_LOOP, "%lld members repeated within a hyperedge", (long long)f[4]);
        return DGEC_OK;
    }
    if (!h.directed) {
        TK(c, "k_h_path", k_h_path<<<grid_for(h.Ms, kBlock, kStreamCap), kBlock, 0, st>>>(S, h.Ms, p.idbits, s.k1));
    } else {
        if (h.Md > 0)
            TK(c, "k_h_type1", k_h_type1<<<grid_for(h.Md, kBlock, kStreamCap), kBlock, 0, st>>>(D, h.Md, S, p.idbits, s.k1));
        if (h.Ms > 0)
            TK(c, "k_h_type2", k_h_type2<<<grid_for(h.Ms, kBlock, kStreamCap), kBlock, 0, st>>>(D, S, h.Ms, h.Md, p.idbits,
                                                                                      s.k1, s.f));
    }
    DG_TRY(read_counters(c, (const int64_t *)s.f, kHFlags, f));
    if (f[4]) return set_err(c, DGEC_ERR_SELF_LOOP, "%lld members repeated within a hyperedge", (long long)f[4]);
    if (f[5])
        return set_err(c, DGEC_ERR_SELF_LOOP, "%lld hyperedges have a vertex as both source and target", (long long)f[5]);
    bool in_b;
    DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, L, 0, 2 * p.idbits, s.radix, &in_b));
    const unsigned long long *lk = in_b ? s.k2 : s.k1;
    TK(c, "k_h_uflag", k_h_uflag<<<grid_for(L + 1, kBlock, kStreamCap), kBlock, 0, st>>>(lk, L, s.flag));
    DG_TRY(exclusive_scan_i32(c, s.flag, s.pos, L + 1, s.scan_tmp));
    TK(c, "k_h_links", k_h_links<<<grid_for(L, kBlock, kStreamCap), kBlock, 0, st>>>(lk, L, s.flag, s.pos, p.idbits,
                                                                               g.orig_of, g.it, sk));
    int64_t n;
    DG_TRY(read_counters(c, (const int64_t *)(s.pos + L), 1, &n));
    sk.n = n;
    return DGEC_OK;
}

}  // namespace dgec

// ------------------------------------------------------------------ C ABI

namespace {

using namespace dgec;

struct HLayout {
    int64_t *eoff, *voff, *knn_off;
    int32_t *gk, *gM, *egraph;
    Csr csr;
    HyperLists S, D;
    Skel skel;
    Msf msf;
    Dendro den;
    Condensed cond;
    void *scratch = nullptr;
    size_t total = 0;
};

Problem hyper_problem(const HyperProblem &h, int32_t M) {
    Problem p;
    p.src = p.dst = nullptr;
    p.t = h.t;
    p.E = h.E;
    p.V = h.V;
    p.k = 1;
    p.M = M;
    p.G = 1;
    p.knn = false;
    p.links_cap = h.directed ? h.Ms + h.Md : h.Ms;
    return p;
}

HLayout plan_hlayout(void *base, const HyperProblem &h, const Problem &p) {
    HLayout L;
    Arena a(base, SIZE_MAX);
    L.eoff = a.take<int64_t>(2);
    L.voff = a.take<int64_t>(2);
    L.knn_off = a.take<int64_t>(2);
    L.gk = a.take<int32_t>(1);
    L.gM = a.take<int32_t>(1);
    L.egraph = a.take<int32_t>(h.E);
    plan_hyper(a, h, L.csr, L.S, L.D, L.skel);
    plan_msf(a, p, L.msf);
    plan_dendro(a, p, L.den);
    plan_condensed(a, p, L.cond);
    size_t scr = std::max({hyper_scratch_bytes(h), msf_scratch_bytes(p), dendro_scratch_bytes(p),
                           condense_scratch_bytes(p)});
    L.scratch = a.take<char>(scr);
    L.total = a.off + 256;
    return L;
}

dgec_status check_hyper(Ctx *c, int64_t E, int32_t V, int64_t Ms, int64_t Md, const dgec_hyper_params *hp) {
    if (!hp) return set_err(c, DGEC_ERR_INVALID_ARG, "params is null");
    if (hp->flags != 0) return set_err(c, DGEC_ERR_INVALID_ARG, "flags must be 0");
    if (hp->directed != 0 && hp->directed != 1) return set_err(c, DGEC_ERR_INVALID_ARG, "directed must be 0 or 1");
    if (hp->min_cluster_size < 2) return set_err(c, DGEC_ERR_INVALID_ARG, "min_cluster_size must be >= 2");
    if (E < 0 || V < 0 || Ms < 0 || Md < 0) return set_err(c, DGEC_ERR_INVALID_ARG, "negative size");
    if (!hp->directed && Md != 0) return set_err(c, DGEC_ERR_INVALID_ARG, "targets given for an undirected hypergraph");
    if (E > 0 && V == 0 && Ms + Md > 0) return set_err(c, DGEC_ERR_VERTEX_RANGE, "members but no vertices");
    if (E >= (int64_t(1) << 30)) return set_err(c, DGEC_ERR_TOO_LARGE, "hyperedges must be < 2^30");
    if (Ms + Md >= (int64_t(1) << 31)) return set_err(c, DGEC_ERR_TOO_LARGE, "members must be < 2^31");
    return DGEC_OK;
}

HyperProblem make_hyper(const int64_t *t, int64_t E, int32_t V, const int64_t *so, const int32_t *sv, int64_t Ms,
                        const int64_t *dofs, const int32_t *dv, int64_t Md, bool directed) {
    HyperProblem h;
    h.t = t;
    h.E = E;
    h.V = V;
    h.s_off = so;
    h.s_vert = sv;
    h.Ms = Ms;
    h.d_off = directed ? dofs : nullptr;
    h.d_vert = directed ? dv : nullptr;
    h.Md = directed ? Md : 0;
    h.directed = directed;
    return h;
}

}  // namespace

extern "C" {

dgec_status dgec_hyper_workspace_size(int64_t n_hyperedges, int32_t n_vertices, int64_t n_src_members,
                                      int64_t n_dst_members, const dgec_hyper_params *params, size_t *bytes) {
    if (!bytes) return DGEC_ERR_INVALID_ARG;
    DG_TRY(check_hyper(nullptr, n_hyperedges, n_vertices, n_src_members, n_dst_members, params));
    HyperProblem h = make_hyper(nullptr, n_hyperedges, n_vertices, nullptr, nullptr, n_src_members, nullptr, nullptr,
                                n_dst_members, params->directed);
    *bytes = plan_hlayout(nullptr, h, hyper_problem(h, params->min_cluster_size)).total;
    return DGEC_OK;
}

dgec_status dgec_run_hyper(dgec_ctx *x, const int64_t *d_t, int64_t n_hyperedges, int32_t n_vertices,
                           const int64_t *d_src_off, const int32_t *d_src_vert, int64_t n_src_members,
                           const int64_t *d_dst_off, const int32_t *d_dst_vert, int64_t n_dst_members,
                           const dgec_hyper_params *params, void *d_ws, size_t ws_bytes, void *stream,
                           dgec_hyper_result *out) {
    if (!x) return DGEC_ERR_INVALID_ARG;
    Ctx *c = &x->c;
    c->msg[0] = 0;
    c->launches = 0;
    if (!out) return set_err(c, DGEC_ERR_INVALID_ARG, "out is null");
    DG_TRY(check_hyper(c, n_hyperedges, n_vertices, n_src_members, n_dst_members, params));
    const bool directed = params->directed;
    if (n_hyperedges > 0 && (!d_t || !d_src_off || (directed && !d_dst_off)))
        return set_err(c, DGEC_ERR_INVALID_ARG, "null input");
    if ((n_src_members > 0 && !d_src_vert) || (n_dst_members > 0 && !d_dst_vert))
        return set_err(c, DGEC_ERR_INVALID_ARG, "null member array");
    if (!d_ws || ((uintptr_t)d_ws & 255))
        return set_err(c, DGEC_ERR_INVALID_ARG, "workspace null or not 256-byte aligned");
    CU_TRY(c, cudaSetDevice(c->device));
    c->stream = (cudaStream_t)stream;
    memset(out, 0, sizeof(*out));
    HyperProblem h = make_hyper(d_t, n_hyperedges, n_vertices, d_src_off, d_src_vert, n_src_members, d_dst_off,
                                d_dst_vert, n_dst_members, directed);
    Problem p = hyper_problem(h, params->min_cluster_size);
    size_t need = plan_hlayout(nullptr, h, p).total;
    if (ws_bytes < need) return set_err(c, DGEC_ERR_OOM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    HLayout L = plan_hlayout(d_ws, h, p);
    // the one-graph tables the shared stages read
    {
        int64_t tab[6] = {0, h.E, 0, h.V, 0, 0};
        int32_t small[2] = {1, params->min_cluster_size};
        CU_TRY(c, cudaMemcpyAsync(L.eoff, tab, sizeof(int64_t) * 2, cudaMemcpyHostToDevice, c->stream));
        CU_TRY(c, cudaMemcpyAsync(L.voff, tab + 2, sizeof(int64_t) * 2, cudaMemcpyHostToDevice, c->stream));
        CU_TRY(c, cudaMemcpyAsync(L.knn_off, tab + 4, sizeof(int64_t) * 2, cudaMemcpyHostToDevice, c->stream));
        CU_TRY(c, cudaMemcpyAsync(L.gk, small, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CU_TRY(c, cudaMemcpyAsync(L.gM, small + 1, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        if (h.E > 0) CU_TRY(c, cudaMemsetAsync(L.egraph, 0, sizeof(int32_t) * h.E, c->stream));
        CU_TRY(c, cudaStreamSynchronize(c->stream));
    }
    p.eoff = L.eoff;
    p.voff = L.voff;
    p.knn_off = L.knn_off;
    p.gk = L.gk;
    p.gM = L.gM;
    p.egraph = L.egraph;
    tl_stream_ctas = c->stream_ctas;
    stage_start(c);
    DG_STAGE("H hypergraph skeleton", stage_hyper(c, p, h, L.csr, L.S, L.D, L.skel, L.scratch));
    DG_STAGE("C spanning forest", stage_msf(c, p, L.csr, L.skel, L.msf, L.scratch));
    DG_STAGE("D1 dendrogram", stage_dendro(c, p, L.csr, L.msf, L.den, L.scratch));
    DG_STAGE("D2 condense and labels", stage_condense(c, p, L.msf, L.den, L.cond, L.scratch));
    CU_TRY(c, cudaStreamSynchronize(c->stream));
    CU_TRY(c, cudaGetLastError());
    kt_collect(c);
    stage_collect(c);
    out->src_voff = L.S.voff;
    out->src_list = L.S.id;
    out->dst_voff = directed ? L.D.voff : nullptr;
    out->dst_list = directed ? L.D.id : nullptr;
    out->sk_u = L.skel.u;
    out->sk_v = L.skel.v;
    out->sk_w = L.skel.w;
    out->mst_u = L.msf.u;
    out->mst_v = L.msf.v;
    out->mst_w = L.msf.w;
    out->link_a = L.den.a;
    out->link_b = L.den.b;
    out->link_size = L.den.size;
    out->labels = L.cond.labels;
    out->n_skeleton = L.skel.n;
    out->n_mst = L.msf.n;
    out->n_clusters = L.cond.n_clusters;
    return DGEC_OK;
}

}  // extern "C"
