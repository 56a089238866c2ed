// Device-wide building blocks: tiled scans, stable LSD radix sort of 64-bit
// keys (with optional 64-bit payloads), stream compaction helpers.
#pragma once

#include "common.cuh"

namespace dgec {

// ------------------------------------------------------------ block scans

template <class T, class Op>
__device__ __forceinline__ T warp_inclusive(T v, Op op) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if ((int)lane_id() >= d) v = op(o, v);
    }
    return v;
}

// Exclusive scan across the CTA (blockDim.x == kBlock). Returns the
// exclusive prefix of v and the CTA total in *total. smem: kBlock/32 slots.
template <class T, class Op>
__device__ __forceinline__ T block_exclusive(T v, Op op, T identity, T *smem, T *total) {
    const int w = threadIdx.x >> 5, nw = kBlock >> 5;
    T inc = warp_inclusive(v, op);
    if (lane_id() == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = (int)lane_id() < nw ? smem[lane_id()] : identity;
        s = warp_inclusive(s, op);
        if ((int)lane_id() < nw) smem[lane_id()] = s;
    }
    __syncthreads();
    T warp_prefix = w > 0 ? smem[w - 1] : identity;
    T excl = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane_id() == 0) excl = identity;
    T res = (w > 0) ? (lane_id() == 0 ? warp_prefix : op(warp_prefix, excl)) : excl;
    *total = smem[nw - 1];
    __syncthreads();
    return res;
}

struct SumI64 {
    __device__ __forceinline__ long long operator()(long long a, long long b) const { return a + b; }
};

// (value, head flag) pairs: a segmented sum where a set flag starts a segment.
struct SegVal {
    long long v;
    int f;
};
struct SegSumOp {
    __device__ __forceinline__ SegVal operator()(SegVal a, SegVal b) const {
        SegVal r;
        r.v = b.f ? b.v : a.v + b.v;
        r.f = a.f | b.f;
        return r;
    }
};

// SegVal shuffles word by word (found by argument-dependent lookup from
// the scan templates above).
__device__ __forceinline__ SegVal __shfl_up_sync(unsigned m, SegVal x, unsigned d) {
    SegVal r;
    r.v = ::__shfl_up_sync(m, x.v, d);
    r.f = ::__shfl_up_sync(m, x.f, d);
    return r;
}

// ----------------------------------------------------- device-wide scans
// Three passes: per-tile aggregates, scan of aggregates (recursive), tile
// scans seeded with their prefix. Works for any associative Op.

template <class T, class Op, class Load>
__global__ void __launch_bounds__(kBlock) k_tile_reduce(Load ld, int64_t n, Op op, T identity,
                                                        T *agg) {
    __shared__ T sm[kBlock / 32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    T acc = identity;
#pragma unroll
    for (int i = 0; i < kItems; i++)
        if (base + i < n) acc = op(acc, ld(base + i));
    T total;
    block_exclusive(acc, op, identity, sm, &total);
    if (threadIdx.x == 0) agg[blockIdx.x] = total;
}

template <class T, class Op, class Load, class Store>
__global__ void __launch_bounds__(kBlock) k_tile_scan(Load ld, Store st, int64_t n, Op op,
                                                      T identity, const T *prefix, bool inclusive) {
    __shared__ T sm[kBlock / 32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    T items[kItems];
    T acc = identity;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        items[i] = (base + i < n) ? ld(base + i) : identity;
        acc = op(acc, items[i]);
    }
    T total;
    T run = block_exclusive(acc, op, identity, sm, &total);
    if (prefix) run = op(prefix[blockIdx.x], run);
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        if (base + i < n) {
            T nxt = op(run, items[i]);
            st(base + i, inclusive ? nxt : run);
            run = nxt;
        }
    }
}

template <class T>
struct LoadPtr {
    const T *p;
    __device__ __forceinline__ T operator()(int64_t i) const { return p[i]; }
};
template <class T>
struct StorePtr {
    T *p;
    __device__ __forceinline__ void operator()(int64_t i, T v) const { p[i] = v; }
};
struct LoadI32AsI64 {
    const int *p;
    __device__ __forceinline__ long long operator()(int64_t i) const { return p[i]; }
};

// Scratch bytes a scan of n items needs (aggregates at every level).
inline size_t scan_scratch_elems(int64_t n) {
    size_t s = 0;
    while (n > kTile) {
        n = cdiv(n, kTile);
        s += (size_t)n * 2 + 64;
    }
    return s + 64;
}

template <class T, class Op, class Load, class Store>
dgec_status device_scan(Ctx *c, Load ld, Store st, int64_t n, Op op, T identity,
                        bool inclusive, T *scratch) {
    if (n <= 0) return DGEC_OK;
    int64_t tiles = cdiv(n, kTile);
    if (tiles == 1) {
        k_tile_scan<T, Op, Load, Store><<<1, kBlock, 0, c->stream>>>(ld, st, n, op, identity,
                                                                     nullptr, inclusive);
        LAUNCH_CHECK(c);
        return DGEC_OK;
    }
    T *agg = scratch;
    T *aggx = scratch + tiles;
    k_tile_reduce<T, Op, Load><<<(unsigned)tiles, kBlock, 0, c->stream>>>(ld, n, op, identity, agg);
    LAUNCH_CHECK(c);
    DG_TRY((device_scan<T, Op, LoadPtr<T>, StorePtr<T>>(c, LoadPtr<T>{agg}, StorePtr<T>{aggx},
                                                        tiles, op, identity, false,
                                                        scratch + 2 * tiles + 32)));
    k_tile_scan<T, Op, Load, Store><<<(unsigned)tiles, kBlock, 0, c->stream>>>(ld, st, n, op,
                                                                               identity, aggx,
                                                                               inclusive);
    LAUNCH_CHECK(c);
    return DGEC_OK;
}

// Exclusive prefix sums to int64 (host wrappers in prims.cu).
dgec_status exclusive_scan_i32(Ctx *c, const int *in, long long *out, int64_t n, long long *scratch);
dgec_status exclusive_scan_i64(Ctx *c, const long long *in, long long *out, int64_t n,
                               long long *scratch);
// Inclusive segmented sum: out[i] = sum of v over [segment start .. i].
dgec_status segmented_inclusive_sum(Ctx *c, const long long *v, const int *head, long long *out,
                                    int64_t n, SegVal *scratch);

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort on key bits [begin_bit, end_bit), 8 bits a pass.
// keys/vals are sorted between (a) and (b) buffers; on return *in_b tells
// which buffer holds the result. vals may be null.
struct RadixBuffers {
    unsigned long long *ka, *kb, *va, *vb;
};
size_t radix_scratch_bytes(int64_t n);
dgec_status radix_sort(Ctx *c, RadixBuffers buf, int64_t n, int begin_bit, int end_bit,
                       void *scratch, bool *in_b);

}  // namespace dgec
