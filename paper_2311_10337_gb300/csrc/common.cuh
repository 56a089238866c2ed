// Shared internals of the dgec CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/dgec.h"

namespace dgec {

constexpr int kBlock = 256;     // threads per CTA for streaming kernels
constexpr int kItems = 8;       // items per thread in tiled kernels
constexpr int kTile = kBlock * kItems;
// Upper bound on any pointer walk in a kernel (the walks follow forests,
// so a bound is never reached on valid state; it only guarantees exit).
constexpr int kMaxWalk = 1 << 26;

// Per-kernel CUDA-event timing: off, one named kernel, or every launch.
constexpr int kMaxTimed = 1 << 14;
constexpr int kMaxNames = 128;
struct KernelTimer {
    int mode = 0;              // 0 off, 1 only `only`, 2 all, 3 names starting with `only`
    char only[64] = {0};
    cudaEvent_t *ev = nullptr;  // 2 * kMaxTimed events, created on first use
    int used = 0;
    int name_of[kMaxTimed];
    const char *names[kMaxNames];
    int n_names = 0;
    double ms[kMaxNames];
    long long count[kMaxNames];
};

// CUDA events at the boundaries of the pipeline stages of the last call
// (always on: a handful of events per call).
constexpr int kMaxStages = 16;
struct StageTimer {
    cudaEvent_t ev[kMaxStages + 1] = {};
    const char *name[kMaxStages] = {};
    float ms[kMaxStages] = {};
    int n = 0;
};

struct Ctx {
    int device = 0;
    int knn_block = 128;           // launch configuration (dgec_set_launch_config)
    int knn_packed = 2;
    int64_t stream_ctas = 65536;
    int num_sms = 152;
    char msg[512] = {0};
    int64_t launches = 0;
    int64_t *h_pinned = nullptr;    // small pinned buffer for counter reads
    cudaStream_t stream = nullptr;
    KernelTimer *kt = nullptr;
    StageTimer stages;
};

void stage_start(Ctx *c);
void stage_mark(Ctx *c, const char *name);
void stage_collect(Ctx *c);

int kt_begin(Ctx *c, const char *name);
void kt_end(Ctx *c, int slot);
void kt_collect(Ctx *c);

dgec_status set_err(Ctx *c, dgec_status s, const char *fmt, ...);

#define DG_TRY(expr)                                   \
    do {                                               \
        dgec_status _s = (expr);                       \
        if (_s != DGEC_OK) return _s;                  \
    } while (0)

// A named range over one pipeline stage on the host timeline (NVTX), for
// profilers that record NVTX ranges; nothing is recorded when none is
// attached. The range closes on every exit, the error returns included.
// A completed stage also records a CUDA event on the call's stream, so the
// device time of every stage of the last call can be read back.
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange &) = delete;
    StageRange &operator=(const StageRange &) = delete;
};

#define DG_STAGE(name, expr)        \
    do {                            \
        StageRange _range(name);    \
        DG_TRY(expr);               \
        ::dgec::stage_mark(c, name); \
    } while (0)

#define CU_TRY(c, expr)                                                          \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess)                                                   \
            return ::dgec::set_err((c), DGEC_ERR_CUDA, "%s:%d %s: %s", __FILE__, \
                                   __LINE__, #expr, cudaGetErrorString(_e));     \
    } while (0)

// Check the last launch (asynchronous errors surface at the next sync).
#define LAUNCH_CHECK(c)                                                           \
    do {                                                                          \
        (c)->launches++;                                                          \
        cudaError_t _e = cudaGetLastError();                                      \
        if (_e != cudaSuccess)                                                    \
            return ::dgec::set_err((c), DGEC_ERR_CUDA, "%s:%d launch: %s", __FILE__, \
                                   __LINE__, cudaGetErrorString(_e));             \
    } while (0)

// Launch a kernel (the variadic part is the whole launch expression),
// bracketed by timing events when timing is on, then check it.
#define TK(c, name, ...)                                  \
    do {                                                  \
        int _slot = ::dgec::kt_begin((c), (name));        \
        __VA_ARGS__;                                      \
        ::dgec::kt_end((c), _slot);                       \
        LAUNCH_CHECK(c);                                  \
    } while (0)

// Bump allocator over the caller's workspace. With base == nullptr it only
// measures, so dgec_workspace_size and dgec_run share one layout.
struct Arena {
    char *base;
    size_t cap;
    size_t off = 0;
    Arena(void *b, size_t c) : base((char *)b), cap(c) {}
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += n * sizeof(T) + 16;
        return p;
    }
    bool ok() const { return off <= cap; }
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// CTA count of the grid-stride streaming kernels launched by this thread's
// current call (set from the context's launch configuration when a call
// starts; each server lane runs its calls on its own thread).
extern thread_local int64_t tl_stream_ctas;
constexpr int64_t kStreamCap = -1;  // max_blocks sentinel: use tl_stream_ctas

inline int grid_for(int64_t n, int block = kBlock, int64_t max_blocks = 1 << 20) {
    if (max_blocks == kStreamCap) max_blocks = tl_stream_ctas;
    int64_t g = cdiv(n, block);
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

inline int bits_for(uint64_t maxval) {  // bits to hold values 0..maxval
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

// Read n int64 counters from device memory (synchronises the stream).
dgec_status read_counters(Ctx *c, const int64_t *d, int n, int64_t *host);

// ---------------------------------------------------------------- device

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned long long atomic_min_u64(unsigned long long *p,
                                                             unsigned long long v) {
    return atomicMin(p, v);
}

// Warp-aggregated increment of counter[key] by 1 per lane; returns this
// lane's slot (old value + rank among lanes with the same key). All lanes
// in `active` must call it.
__device__ __forceinline__ int warp_agg_inc(int *counter, int key, unsigned active) {
    unsigned peers = __match_any_sync(active, key);
    int leader = __ffs(peers) - 1;
    unsigned lt = peers & ((1u << lane_id()) - 1u);
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(&counter[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(lt);
}

// Stream compaction slot through ONE atomicAdd per CTA: threads with
// `take` get consecutive slots of `counter` (order within the CTA follows
// thread order). Every thread of the CTA must call it the same number of
// times (use CTA-uniform loops).
__device__ __forceinline__ long long cta_reserve(bool take, unsigned long long *counter) {
    __shared__ unsigned s_warp[32];
    __shared__ unsigned long long s_base;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane_id() == 0) s_warp[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int i = 0; i < nw; i++) {
            unsigned c = s_warp[i];
            s_warp[i] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(counter, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    long long slot = (long long)(s_base + s_warp[w] + __popc(m & ((1u << lane_id()) - 1u)));
    __syncthreads();
    return slot;
}

// Stream compaction with one atomicAdd per CTA for up to blockDim.x * 32
// items: thread i asks for cnt_i slots and gets the first of its own
// consecutive run (runs in thread order). Every thread of the CTA must call
// it the same number of times (use CTA-uniform loops).
__device__ __forceinline__ long long cta_reserve_count(unsigned cnt, unsigned long long *counter) {
    __shared__ unsigned s_warp[32];
    __shared__ unsigned long long s_base;
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    unsigned inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
        if ((int)lane_id() >= d) inc += o;
    }
    if (lane_id() == 31) s_warp[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int i = 0; i < nw; i++) {
            const unsigned c = s_warp[i];
            s_warp[i] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(counter, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    const long long slot = (long long)(s_base + s_warp[w] + inc - cnt);
    __syncthreads();
    return slot;
}

// 128-bit unsigned add into (hi, lo) words; exact and order independent.
__device__ __forceinline__ void atomic_add_u128(unsigned long long *hi,
                                                unsigned long long *lo,
                                                unsigned long long add_hi,
                                                unsigned long long add_lo) {
    unsigned long long old = atomicAdd(lo, add_lo);
    unsigned long long carry = (old + add_lo < old) ? 1ull : 0ull;
    if (add_hi | carry) atomicAdd(hi, add_hi + carry);
}

// Adds the `val` (below 2^96) of every lane in `active` with `has` set to
// the 128-bit counter (hi[key], lo[key]), summing lanes that share a key
// first (one atomic pair per distinct key per warp). The sum is exact: values
// are split into six 16-bit limbs whose warp sums fit in 32 bits. All lanes
// in `active` must call it.
__device__ __forceinline__ void warp_add_u96(unsigned active, bool has, int key, unsigned __int128 val,
                                             unsigned long long *hi, unsigned long long *lo) {
    const unsigned peers = __match_any_sync(active, has ? key : -1);
    if (!has) return;
    unsigned s[6];
#pragma unroll
    for (int i = 0; i < 6; i++) s[i] = __reduce_add_sync(peers, (unsigned)(val >> (16 * i)) & 0xffffu);
    if ((int)lane_id() == __ffs(peers) - 1) {
        unsigned __int128 tot = 0;
#pragma unroll
        for (int i = 0; i < 6; i++) tot += (unsigned __int128)s[i] << (16 * i);
        atomic_add_u128(&hi[key], &lo[key], (unsigned long long)(tot >> 64), (unsigned long long)tot);
    }
}

// lambda(w) = floor((2^64 - 1) / (w + 1)) for w >= 0; 0 stands for w = inf.
__device__ __forceinline__ unsigned long long lambda_of(long long w) {
    return 0xFFFFFFFFFFFFFFFFull / ((unsigned long long)w + 1ull);
}

}  // namespace dgec

// The C ABI's context handle wraps one internal context.
struct dgec_ctx {
    dgec::Ctx c;
};
