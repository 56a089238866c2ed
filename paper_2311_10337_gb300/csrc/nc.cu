// Stage N (optional): the nearly-causal line graph of Sec. 4.3, where an arc
// r -> s (dst r = src s) may also point up to delta back in time
// (t_s >= t_r - delta), weighed |t_s - t_r|. At a vertex its arcs are the
// causal ones (Def. 1) and the backward ones (t_s < t_r <= t_s + delta).
// An MST of a union of two graphs lies in the union of their MSTs; Alg. 2
// gives the causal part's (Thm. 2); on the graph with negated times Alg. 2
// gives the MST of all backward pairs, and its links with w <= delta are the
// MSF of the capped family (Kruskal stopped at delta). So the skeleton is
// L*(G) together with the links of L*(G with -t) of weight <= delta, kept
// once; stages A and B simply run a second time on the negated times.
//
// The kNN lists merge likewise: the candidates of e are its causal ones and
// its backward ones (the causal candidates of the negated graph) within
// delta, both already ranked by (|dt|, id); the merge keeps the first k
// distinct ids (a concurrent edge sits in both and counts once).
#include "stages.cuh"

namespace dgec {

__global__ void k_nc_negate(const int64_t *t, int64_t E, int64_t *tn) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        tn[e] = -t[e];
}

__global__ void k_nc_keys(const int32_t *u1, const int32_t *v1, int64_t n1, const int32_t *u2, const int32_t *v2,
                          const int64_t *w2, int64_t n2, int64_t dnc, int idbits, unsigned long long *key) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n1 + n2;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = ~0ull;
        if (x < n1) {
            k = ((unsigned long long)(unsigned)u1[x] << idbits) | (unsigned)v1[x];
        } else {
            const int64_t y = x - n1;
            if (w2[y] <= dnc) k = ((unsigned long long)(unsigned)u2[y] << idbits) | (unsigned)v2[y];
        }
        key[x] = k;
    }
}

__global__ void k_nc_flag(const unsigned long long *key, int64_t L, int *flag) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= L;
         x += (int64_t)gridDim.x * blockDim.x)
        flag[x] = x < L && key[x] != ~0ull && (x == 0 || key[x] != key[x - 1]);
}

__global__ void k_nc_emit(const unsigned long long *key, int64_t L, const int *flag, const long long *pos, int idbits,
                          const int32_t *rank_of, const int64_t *t, Skel h) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[x]) continue;
        const int u = (int)(key[x] >> idbits), v = (int)(key[x] & ((1ull << idbits) - 1ull));
        const int64_t at = pos[x];
        h.u[at] = u;
        h.v[at] = v;
        h.ru[at] = rank_of[u];
        h.rv[at] = rank_of[v];
        const long long d = t[u] - t[v];
        h.w[at] = d < 0 ? -d : d;
    }
}

// Merge the causal row a and the backward row b (entries of b beyond delta
// end it) of every edge, by (|dt|, id), first k distinct ids.
__global__ void k_nc_knn(int64_t E, int k, const int64_t *t, const int32_t *ka, const int32_t *kb, int64_t dnc,
                         int32_t *out, int64_t *core) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *ra = ka + e * k, *rb = kb + e * k;
        int32_t *ro = out + e * k;
        const long long te = t[e];
        int i = 0, j = 0, cnt = 0, last = -1;
        long long lastw = LLONG_MAX;
        auto wt = [&](int id) -> long long {
            const long long d = t[id] - te;
            return d < 0 ? -d : d;
        };
        int ida = i < k ? ra[i] : -1, idb = j < k ? rb[j] : -1;
        long long wa = ida >= 0 ? wt(ida) : LLONG_MAX, wb = idb >= 0 ? wt(idb) : LLONG_MAX;
        if (wb > dnc) idb = -1;
        for (int step = 0; step < 2 * k && cnt < k && (ida >= 0 || idb >= 0); step++) {
            const bool take_a = idb < 0 || (ida >= 0 && (wa < wb || (wa == wb && ida <= idb)));
            int id;
            long long w;
            if (take_a) {
                id = ida;
                w = wa;
                i++;
                ida = i < k ? ra[i] : -1;
                wa = ida >= 0 ? wt(ida) : LLONG_MAX;
            } else {
                id = idb;
                w = wb;
                j++;
                idb = j < k ? rb[j] : -1;
                wb = idb >= 0 ? wt(idb) : LLONG_MAX;
                if (wb > dnc) idb = -1;
            }
            if (id != last) {
                ro[cnt++] = id;
                last = id;
                lastw = w;
            }
        }
        for (int x = cnt; x < k; x++) ro[x] = -1;
        core[e] = cnt == k ? lastw : LLONG_MAX;
    }
}

void plan_nc(Arena &ws, const Problem &p, Skel &h) {
    const int64_t L = 4 * p.E;  // both skeletons
    h.u = ws.take<int32_t>(L);
    h.v = ws.take<int32_t>(L);
    h.ru = ws.take<int32_t>(L);
    h.rv = ws.take<int32_t>(L);
    h.w = ws.take<int64_t>(L);
    h.knn = ws.take<int32_t>(p.E * (int64_t)p.k);
    h.core = ws.take<int64_t>(p.E);
    h.n = 0;
}

struct NcScratch {
    unsigned long long *k1, *k2;
    int *flag;
    long long *pos, *scan_tmp;
    void *radix;
};
static NcScratch carve_nc(Arena &a, const Problem &p) {
    NcScratch s;
    const int64_t L = 4 * p.E > 0 ? 4 * p.E : 1;
    s.k1 = a.take<unsigned long long>(L);
    s.k2 = a.take<unsigned long long>(L);
    s.flag = a.take<int>(L + 1);
    s.pos = a.take<long long>(L + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(L + 1));
    s.radix = a.take<char>(radix_scratch_bytes(L));
    return s;
}
size_t nc_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_nc(a, p);
    return a.off;
}

dgec_status stage_nc_negate(Ctx *c, const Problem &p, int64_t *tn) {
    if (p.E > 0)
        TK(c, "k_nc_negate", k_nc_negate<<<grid_for(p.E, kBlock, kStreamCap), kBlock, 0, c->stream>>>(p.t, p.E, tn));
    return DGEC_OK;
}

dgec_status stage_nc(Ctx *c, const Problem &p, const Csr &g, const Skel &s1, const Skel &s2, Skel &h,
                     void *scratch) {
    cudaStream_t st = c->stream;
    h.n = 0;
    const int64_t E = p.E, L = s1.n + s2.n;
    if (E == 0) return DGEC_OK;
    if (L > 4 * E) return set_err(c, DGEC_ERR_INTERNAL, "nearly-causal skeleton over capacity");
    Arena a(scratch, SIZE_MAX);
    NcScratch s = carve_nc(a, p);
    TK(c, "k_nc_knn", k_nc_knn<<<grid_for(E, kBlock, kStreamCap), kBlock, 0, st>>>(E, p.k, p.t, s1.knn, s2.knn, p.dnc,
                                                                             h.knn, h.core));
    if (L == 0) return DGEC_OK;
    const int gL = grid_for(L, kBlock, kStreamCap);
    TK(c, "k_nc_keys", k_nc_keys<<<gL, kBlock, 0, st>>>(s1.u, s1.v, s1.n, s2.u, s2.v, s2.w, s2.n, p.dnc, p.idbits,
                                                       s.k1));
    bool in_b;
    DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, L, 0, 2 * p.idbits, s.radix, &in_b));
    const unsigned long long *key = in_b ? s.k2 : s.k1;
    TK(c, "k_nc_flag", k_nc_flag<<<grid_for(L + 1, kBlock, kStreamCap), kBlock, 0, st>>>(key, L, s.flag));
    DG_TRY(exclusive_scan_i32(c, s.flag, s.pos, L + 1, s.scan_tmp));
    TK(c, "k_nc_emit", k_nc_emit<<<gL, kBlock, 0, st>>>(key, L, s.flag, s.pos, p.idbits, g.rank_of, p.t, h));
    int64_t n;
    DG_TRY(read_counters(c, (const int64_t *)(s.pos + L), 1, &n));
    h.n = n;
    return DGEC_OK;
}

}  // namespace dgec
