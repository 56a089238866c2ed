// Stage M (optional): the mutual-reachability graph. An approximation, not
// in the paper: HDBSCAN's mutual reachability weights max(core_a, core_b,
// |dt|) do not keep Thm. 3 (a skeleton path can pass through edges whose
// core distance is larger than the direct arc's), so the graph is widened
// with every edge's kNN pairs: H = L* together with {(e, n) : n in kNN(e)},
// each pair once. Pairs with an endpoint of infinite core (fewer than k
// neighbours) are dropped. The forest, dendrogram and condense stages then
// run on H in place of L*.
//
// Every candidate pair is keyed (min r, max r) in internal ids; one radix
// sort over 2 * idbits bits brings duplicates together, and a flag pass
// keeps the first of each run whose weight is finite; a scan compacts.
#include "stages.cuh"

namespace dgec {

__device__ __forceinline__ unsigned long long mrd_key(int a, int b, int idbits) {
    const unsigned long long lo = (unsigned)(a < b ? a : b), hi = (unsigned)(a < b ? b : a);
    return (lo << idbits) | hi;
}

__global__ void k_mrd_keys(const int32_t *ru, const int32_t *rv, int64_t n, const int32_t *knn, int64_t E, int k,
                           const int32_t *rank_of, int idbits, unsigned long long *key) {
    const int64_t L = n + E * (int64_t)k;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long kk = ~0ull;
        if (x < n) {
            kk = mrd_key(ru[x], rv[x], idbits);
        } else {
            const int64_t y = x - n;
            const int nb = knn[y];
            if (nb >= 0) kk = mrd_key(rank_of[y / k], rank_of[nb], idbits);
        }
        key[x] = kk;
    }
}

__device__ __forceinline__ long long mrd_weight(unsigned long long kk, int idbits, const int32_t *orig_of,
                                                const int64_t *it, const int64_t *core, int *ea, int *eb) {
    const int a = (int)(kk >> idbits), b = (int)(kk & ((1ull << idbits) - 1ull));  // a < b: t_a <= t_b
    *ea = orig_of[a];
    *eb = orig_of[b];
    long long m = it[b] - it[a];
    const long long ca = core[*ea], cb = core[*eb];
    if (ca > m) m = ca;
    if (cb > m) m = cb;
    return m;
}

__global__ void k_mrd_flag(const unsigned long long *key, int64_t L, int idbits, const int32_t *orig_of,
                           const int64_t *it, const int64_t *core, int *flag) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= L;
         x += (int64_t)gridDim.x * blockDim.x) {
        int f = 0;
        if (x < L && key[x] != ~0ull && (x == 0 || key[x] != key[x - 1])) {
            int ea, eb;
            f = mrd_weight(key[x], idbits, orig_of, it, core, &ea, &eb) != LLONG_MAX;
        }
        flag[x] = f;
    }
}

__global__ void k_mrd_emit(const unsigned long long *key, int64_t L, const int *flag, const long long *pos,
                           int idbits, const int32_t *orig_of, const int64_t *it, const int64_t *core, Skel h) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[x]) continue;
        int ea, eb;
        const long long m = mrd_weight(key[x], idbits, orig_of, it, core, &ea, &eb);
        const int64_t at = pos[x];
        h.ru[at] = (int)(key[x] >> idbits);
        h.rv[at] = (int)(key[x] & ((1ull << idbits) - 1ull));
        h.u[at] = ea < eb ? ea : eb;
        h.v[at] = ea < eb ? eb : ea;
        h.w[at] = m;
    }
}

void plan_mrd(Arena &ws, const Problem &p, Skel &h) {
    const int64_t L = link_cap(p);
    h.u = ws.take<int32_t>(L);
    h.v = ws.take<int32_t>(L);
    h.ru = ws.take<int32_t>(L);
    h.rv = ws.take<int32_t>(L);
    h.w = ws.take<int64_t>(L);
    h.knn = nullptr;
    h.core = nullptr;
    h.n = 0;
}

struct MrdScratch {
    unsigned long long *k1, *k2;
    int *flag;
    long long *pos, *scan_tmp;
    void *radix;
};
static MrdScratch carve_mrd(Arena &a, const Problem &p) {
    MrdScratch s;
    const int64_t L = link_cap(p) > 0 ? link_cap(p) : 1;
    s.k1 = a.take<unsigned long long>(L);
    s.k2 = a.take<unsigned long long>(L);
    s.flag = a.take<int>(L + 1);
    s.pos = a.take<long long>(L + 1);
    s.scan_tmp = a.take<long long>(scan_scratch_elems(L + 1));
    s.radix = a.take<char>(radix_scratch_bytes(L));
    return s;
}
size_t mrd_scratch_bytes(const Problem &p) {
    Arena a(nullptr, 0);
    carve_mrd(a, p);
    return a.off;
}

dgec_status stage_mrd(Ctx *c, const Problem &p, const Csr &g, const Skel &sk, Skel &h, void *scratch) {
    cudaStream_t st = c->stream;
    h.n = 0;
    const int64_t E = p.E, L = sk.n + E * (int64_t)p.k;
    if (E == 0 || L == 0) return DGEC_OK;
    if (L > link_cap(p)) return set_err(c, DGEC_ERR_INTERNAL, "mutual-reachability graph over capacity");
    Arena a(scratch, SIZE_MAX);
    MrdScratch s = carve_mrd(a, p);
    const int gL = grid_for(L, kBlock, kStreamCap);
    TK(c, "k_mrd_keys", k_mrd_keys<<<gL, kBlock, 0, st>>>(sk.ru, sk.rv, sk.n, sk.knn, E, p.k, g.rank_of, p.idbits,
                                                         s.k1));
    bool in_b;
    DG_TRY(radix_sort(c, RadixBuffers{s.k1, s.k2, nullptr, nullptr}, L, 0, 2 * p.idbits, s.radix, &in_b));
    const unsigned long long *key = in_b ? s.k2 : s.k1;
    TK(c, "k_mrd_flag", k_mrd_flag<<<grid_for(L + 1, kBlock, kStreamCap), kBlock, 0, st>>>(key, L, p.idbits, g.orig_of,
                                                                                    g.it, sk.core, s.flag));
    DG_TRY(exclusive_scan_i32(c, s.flag, s.pos, L + 1, s.scan_tmp));
    TK(c, "k_mrd_emit", k_mrd_emit<<<gL, kBlock, 0, st>>>(key, L, s.flag, s.pos, p.idbits, g.orig_of, g.it, sk.core,
                                                         h));
    int64_t n;
    DG_TRY(read_counters(c, (const int64_t *)(s.pos + L), 1, &n));
    h.n = n;
    return DGEC_OK;
}

}  // namespace dgec
