// Device-wide scans and the stable LSD radix sort.
#include "prims.cuh"

namespace dgec {

dgec_status exclusive_scan_i32(Ctx *c, const int *in, long long *out, int64_t n,
                               long long *scratch) {
    return device_scan<long long, SumI64, LoadI32AsI64, StorePtr<long long>>(
        c, LoadI32AsI64{in}, StorePtr<long long>{out}, n, SumI64{}, 0ll, false, scratch);
}

dgec_status exclusive_scan_i64(Ctx *c, const long long *in, long long *out, int64_t n,
                               long long *scratch) {
    return device_scan<long long, SumI64, LoadPtr<long long>, StorePtr<long long>>(
        c, LoadPtr<long long>{in}, StorePtr<long long>{out}, n, SumI64{}, 0ll, false, scratch);
}

struct LoadSeg {
    const long long *v;
    const int *h;
    __device__ __forceinline__ SegVal operator()(int64_t i) const {
        SegVal s;
        s.v = v[i];
        s.f = h[i];
        return s;
    }
};
struct StoreSeg {
    long long *o;
    __device__ __forceinline__ void operator()(int64_t i, SegVal s) const { o[i] = s.v; }
};

dgec_status segmented_inclusive_sum(Ctx *c, const long long *v, const int *head, long long *out,
                                    int64_t n, SegVal *scratch) {
    SegVal id;
    id.v = 0;
    id.f = 0;
    return device_scan<SegVal, SegSumOp, LoadSeg, StoreSeg>(c, LoadSeg{v, head}, StoreSeg{out}, n,
                                                            SegSumOp{}, id, true, scratch);
}

// ------------------------------------------------------------ radix sort
// One pass = digit histogram per tile, exclusive scan of the digit-major
// [256][tiles] table, then a stable scatter: each warp ranks its 256 keys
// with match_any (keys in position order), the CTA combines warp counts,
// stages the tile in shared memory in digit order and writes it out so
// that runs of one digit land contiguously.

constexpr int kRadix = 256;
struct AddI {
    __device__ __forceinline__ int operator()(int a, int b) const { return a + b; }
};
constexpr int kWarps = kBlock / 32;

__global__ void __launch_bounds__(kBlock) k_radix_hist(const unsigned long long *keys, int64_t n,
                                                       int shift, unsigned mask, int *hist,
                                                       int64_t tiles) {
    __shared__ int cnt[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kBlock) cnt[i] = 0;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    // all loads first, then the counting
    int d[kItems];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        const int64_t idx = base + j * kBlock + threadIdx.x;
        d[j] = idx < n ? (int)((keys[idx] >> shift) & mask) : kRadix;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; j++)
        if (d[j] < kRadix) atomicAdd(&cnt[d[j]], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += kBlock) hist[(int64_t)i * tiles + blockIdx.x] = cnt[i];
}

template <bool VALS>
__global__ void __launch_bounds__(kBlock, 4) k_radix_scatter(
    const unsigned long long *kin, const unsigned long long *vin, unsigned long long *kout,
    unsigned long long *vout, int64_t n, int shift, unsigned mask, const long long *offs,
    int64_t tiles) {
    __shared__ unsigned long long skeys[kTile];
    __shared__ unsigned long long svals[VALS ? kTile : 1];
    __shared__ int wcnt[kWarps][kRadix];
    __shared__ int dstart[kRadix];
    __shared__ long long soff[kRadix];
    __shared__ int scan_sm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kBlock) (&wcnt[0][0])[i] = 0;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    // this tile's global start of digit threadIdx.x (kBlock == kRadix): it
    // does not depend on the keys, so its load overlaps theirs
    const long long gstart = offs[(int64_t)threadIdx.x * tiles + blockIdx.x];
    unsigned long long k[kItems], v[kItems];
    int r[kItems];  // rank among the warp's items of its digit; -1 past the end
    const int64_t wbase = base + warp * (32 * kItems) + lane;
    const int nv = n - wbase > 0 ? (int)((n - wbase + 31) >> 5) : 0;  // this lane's valid items
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const bool ok = i < nv;
        k[i] = ok ? kin[wbase + i * 32] : 0ull;
        if (VALS) v[i] = ok ? vin[wbase + i * 32] : 0ull;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        // the digit is recomputed from the key where needed (fewer live registers)
        const int d = i < nv ? (int)((k[i] >> shift) & mask) : kRadix;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        int before = d < kRadix ? wcnt[warp][d] : 0;
        r[i] = d < kRadix ? before + __popc(peers & lt) : -1;
        __syncwarp();
        if (lane == leader && d < kRadix) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets, tile total; then digit starts in the tile
    int digit = threadIdx.x;  // kBlock == kRadix
    int run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
        int cnt = wcnt[w][digit];
        wcnt[w][digit] = run;
        run += cnt;
    }
    int total;
    int start = block_exclusive(run, AddI{}, 0, scan_sm, &total);
    dstart[digit] = start;
    // this tile's global start of every digit, less its start in the tile
    soff[digit] = gstart - start;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        if (r[i] >= 0) {
            const int d = (int)((k[i] >> shift) & mask);
            int lpos = dstart[d] + wcnt[warp][d] + r[i];
            skeys[lpos] = k[i];
            if (VALS) svals[lpos] = v[i];
        }
    }
    __syncthreads();
    int64_t m = n - base < kTile ? n - base : kTile;
    for (int j = threadIdx.x; j < m; j += kBlock) {
        const unsigned long long key = skeys[j];
        const int dd = (int)((key >> shift) & mask);
        const int64_t g = soff[dd] + j;
        kout[g] = key;
        if (VALS) vout[g] = svals[j];
    }
}

// Small inputs (n <= kSmallSort): one CTA sorts the pairs (key bits
// [begin, end), input position) by a bitonic network in shared memory --
// the same stable order as the LSD passes -- and gathers keys and values
// into the second buffers. One launch instead of five per 8-bit pass.
constexpr int kSmallSort = 2048;
__global__ void __launch_bounds__(1024) k_sort_small(const unsigned long long *kin, const unsigned long long *vin,
                                                     unsigned long long *kout, unsigned long long *vout, int n,
                                                     int begin_bit, int end_bit) {
    __shared__ unsigned long long sf[kSmallSort];
    __shared__ int si[kSmallSort];
    const int nb = end_bit - begin_bit;
    const unsigned long long fmask = nb >= 64 ? ~0ull : ((1ull << nb) - 1ull);
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        sf[i] = i < n ? (kin[i] >> begin_bit) & fmask : ~0ull;
        si[i] = i < n ? i : kSmallSort + i;  // padding sorts last
    }
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long fa = sf[lo], fb = sf[hi];
                const int ia = si[lo], ib = si[hi];
                const bool greater = fa > fb || (fa == fb && ia > ib);
                if (greater == up) {
                    sf[lo] = fb;
                    sf[hi] = fa;
                    si[lo] = ib;
                    si[hi] = ia;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        kout[i] = kin[si[i]];
        if (vin) vout[i] = vin[si[i]];
    }
}

size_t radix_scratch_bytes(int64_t n) {
    int64_t tiles = cdiv(n > 0 ? n : 1, kTile);
    size_t hist = (size_t)tiles * kRadix;
    return hist * sizeof(int) + hist * sizeof(long long) + scan_scratch_elems(hist) * sizeof(long long) +
           1024;
}

dgec_status radix_sort(Ctx *c, RadixBuffers buf, int64_t n, int begin_bit, int end_bit,
                       void *scratch, bool *in_b) {
    *in_b = false;
    if (n <= 1 || end_bit <= begin_bit) return DGEC_OK;
    if (n <= kSmallSort) {
        TK(c, "k_sort_small", k_sort_small<<<1, 1024, 0, c->stream>>>(buf.ka, buf.va, buf.kb, buf.vb, (int)n,
                                                                      begin_bit, end_bit));
        *in_b = true;
        return DGEC_OK;
    }
    int64_t tiles = cdiv(n, kTile);
    size_t hist_n = (size_t)tiles * kRadix;
    char *s = (char *)scratch;
    int *hist = (int *)s;
    s += ((hist_n * sizeof(int) + 255) & ~(size_t)255);
    long long *offs = (long long *)s;
    s += ((hist_n * sizeof(long long) + 255) & ~(size_t)255);
    long long *scan_tmp = (long long *)s;
    unsigned long long *kin = buf.ka, *kout = buf.kb, *vin = buf.va, *vout = buf.vb;
    bool cur_b = false;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        int nb = end_bit - shift < 8 ? end_bit - shift : 8;
        unsigned mask = (1u << nb) - 1u;
        TK(c, "k_radix_hist", k_radix_hist<<<(unsigned)tiles, kBlock, 0, c->stream>>>(kin, n, shift, mask, hist, tiles));
        DG_TRY(exclusive_scan_i32(c, hist, offs, (int64_t)hist_n, scan_tmp));
        if (vin) {
            TK(c, "k_radix_scatter", k_radix_scatter<true><<<(unsigned)tiles, kBlock, 0, c->stream>>>(
                                         kin, vin, kout, vout, n, shift, mask, offs, tiles));
        } else {
            TK(c, "k_radix_scatter", k_radix_scatter<false><<<(unsigned)tiles, kBlock, 0, c->stream>>>(
                                         kin, nullptr, kout, nullptr, n, shift, mask, offs, tiles));
        }
        unsigned long long *t = kin;
        kin = kout;
        kout = t;
        t = vin;
        vin = vout;
        vout = t;
        cur_b = !cur_b;
    }
    *in_b = cur_b;
    return DGEC_OK;
}

}  // namespace dgec
