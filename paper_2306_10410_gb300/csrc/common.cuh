// Device helpers shared by the BOBA kernels: status reporting, streaming
// memory access, block scans and the decoupled look-back prefix used by every
// single-pass scan in this library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/boba.h"

namespace boba {

constexpr uint32_t kSent = 0xFFFFFFFFu;       // key of a vertex on no edge ("infinity")
constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// status word: one bit per boba_status_t code, OR-ed by any kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(uint32_t *st, boba_status_t code)
{
    atomicOr(st, 1u << (int)code);
}

// ---------------------------------------------------------------------------
// memory access with cache hints
// ---------------------------------------------------------------------------
// Edge streams are touched once: load/store them evict-first so that the
// n-sized key/label arrays gathered at random stay resident in L2.
__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(int4 *p, int4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(int *p, int v) { __stcs(p, v); }

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one uint32 per thread (blockDim.x == BLOCK);
// Op is + (default) or max, both with identity 0.
// ---------------------------------------------------------------------------
struct OpSum32 {
    __device__ __forceinline__ static uint32_t apply(uint32_t a, uint32_t b) { return a + b; }
};
struct OpMax32 {
    __device__ __forceinline__ static uint32_t apply(uint32_t a, uint32_t b) { return a > b ? a : b; }
};

template <int BLOCK, class Op = OpSum32>
struct BlockScan {
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    static constexpr int kWarps = BLOCK / 32;
    struct Smem {
        uint32_t warp_sums[kWarps];
        uint32_t total;
    };

    // Returns the exclusive prefix of `x` over the block and writes the block
    // total to *total (all threads).  Contains __syncthreads().
    __device__ __forceinline__ static uint32_t exclusive(uint32_t x, uint32_t *total, Smem &sm)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc = Op::apply(inc, y);
        }
        uint32_t exc = __shfl_up_sync(kFull, inc, 1);
        if (lane == 0) exc = 0;
        if (lane == 31) sm.warp_sums[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < kWarps ? sm.warp_sums[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi = Op::apply(wi, y);
            }
            uint32_t we = __shfl_up_sync(kFull, wi, 1);
            if (lane == 0) we = 0;
            if (lane < kWarps) sm.warp_sums[lane] = we;   // exclusive warp offsets
            if (lane == 31) sm.total = wi;
        }
        __syncthreads();
        const uint32_t r = Op::apply(sm.warp_sums[warp], exc);
        *total = sm.total;
        return r;
    }
};

// ---------------------------------------------------------------------------
// Decoupled look-back (Merrill and Garland, "Single-pass parallel prefix scan
// with decoupled look-back", NVIDIA tech report NVR-2016-002).
//
// One 64-bit status word per tile: the top two bits are the flag (0 = not
// ready, 1 = tile aggregate published, 2 = inclusive prefix published), the
// low 62 bits the value.  Flag and value share one single-copy-atomic word,
// so relaxed loads and stores suffice.  Tiles must be claimed in increasing
// order by running blocks (an atomic ticket), so every tile waited on belongs
// to a block that is already resident: the wait always ends.  It is bounded
// anyway: after kTimeoutNs the tile records BOBA_ERR_TIMEOUT, stops waiting
// and continues with an incomplete prefix.
// ---------------------------------------------------------------------------
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr uint64_t kFlagMask = 3ull << 62;
constexpr uint64_t kValMask = ~kFlagMask;
constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s
constexpr uint32_t kMaxSpins = 1u << 26;          // second bound, independent of the timer

struct OpSum {
    __device__ __forceinline__ static uint64_t apply(uint64_t a, uint64_t b) { return a + b; }
};
struct OpMax {
    __device__ __forceinline__ static uint64_t apply(uint64_t a, uint64_t b) { return a > b ? a : b; }
};

// Called by all 32 lanes of ONE warp.  Returns the exclusive prefix of tile
// `tile` under Op (same value in every lane; the identity, 0, for tile 0) and
// publishes its inclusive prefix.  Values must fit in 62 bits.
// `seg_first` marks the first tile of a segment: it publishes its inclusive
// prefix at once, and no look-back walks past it (segmented scans).
template <class Op = OpSum>
__device__ __forceinline__ uint64_t lookback_exclusive(uint64_t *tstat, int64_t tile, uint64_t agg,
                                                       uint32_t *status, bool seg_first = false,
                                                       uint64_t timeout_ns = kTimeoutNs)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0 || seg_first) {
        if (lane == 0) st_relaxed_u64(&tstat[tile], kFlagPre | agg);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(&tstat[tile], kFlagAgg | agg);
    uint64_t prefix = 0;
    int64_t base = tile - 1;
    uint64_t t0 = 0;
    uint32_t spins = 0;
    bool timed_out = false;
    while (true) {
        const int64_t t = base - lane;
        uint64_t s;
        while (true) {
            s = (t >= 0) ? ld_relaxed_u64(&tstat[t]) : kFlagPre;
            if (__all_sync(kFull, (s & kFlagMask) != 0)) break;
            if (timed_out) { if ((s & kFlagMask) == 0) s = kFlagPre; break; }
            ++spins;
            if ((spins & 255u) == 1u || spins >= kMaxSpins) {
                // lane 0's clock, broadcast, keeps the decision warp-uniform
                const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
                if (t0 == 0) t0 = now;
                if (now - t0 > timeout_ns || spins >= kMaxSpins) {
                    if (lane == 0) raise_status(status, BOBA_ERR_TIMEOUT);
                    timed_out = true;
                }
            }
            __nanosleep(64);
        }
        const unsigned pre = __ballot_sync(kFull, (s & kFlagMask) == kFlagPre);
        const int first = pre ? (__ffs(pre) - 1) : 31;
        uint64_t c = (lane <= first) ? (s & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c = Op::apply(c, __shfl_xor_sync(kFull, c, o));
        prefix = Op::apply(prefix, c);
        if (pre) break;
        base -= 32;
    }
    if (lane == 0) st_relaxed_u64(&tstat[tile], kFlagPre | (Op::apply(prefix, agg) & kValMask));
    return prefix;
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace boba
