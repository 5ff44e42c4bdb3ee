// The two lookup passes of the reorder with their edge streams moved by the
// TMA engine (tuner variant 7 of the first-occurrence and relabel kernels).
//
// k_first (Alg. 2 with AtomicMin, Sec. 4.4) and k_relabel (Sec. 5.3) each read
// the endpoints as a stream and look up one entry of an n-sized array per
// endpoint at a random index.  The lookups are bound by the L1TEX/L2 request
// rate; in the plain kernels the stream's int4 loads (and the relabel's int4
// stores) go through L1TEX beside them.  Here a persistent CTA moves its
// tiles of the stream with bulk asynchronous copies between global and
// shared memory (cp.async.bulk, completion counted on an mbarrier for loads,
// bulk groups for stores), so L1TEX carries only the lookups.
//
// Each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... in increasing
// order through a ring of kTmaBufs shared buffers: the tile k + kTmaBufs is
// loaded as soon as tile k's buffer is free.  In the relabel the labels are
// written over the tile in shared memory and the tile is stored back with a
// bulk copy; a buffer is refilled only once its store has read it.
//
// Tiles cover the first 4 * floor(m / 4) elements of each half of I ++ J (all
// bulk copies are multiples of 16 bytes at 16-byte-aligned addresses; the
// vector path requires aligned arrays); block 0 handles the up to 3 elements
// left in each half.  Every mbarrier wait is bounded: after kTmaSpinLimit
// polls the CTA records BOBA_ERR_TIMEOUT, stops processing, waits (again
// bounded) for the copies it issued and returns.
#include "common.cuh"
#include "host.hpp"
#include "reorder_kernels.cuh"

namespace boba {

constexpr int kTmaBlock = 256;
constexpr int kTmaTile = 4096;                 // elements (16 KB) per tile
constexpr int kTmaBufs = 3;
constexpr size_t kTmaSmem = (size_t)kTmaBufs * kTmaTile * 4;
constexpr uint32_t kTmaSpinLimit = 1u << 26;

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Bounded wait for phase `parity` of the barrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t spin = 0; spin < kTmaSpinLimit; ++spin) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Thread 0: load `bytes` (a multiple of 16) from global `src` into shared
// `dst`, completion counted on `bar`.
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                         uint64_t pol)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Thread 0: store `bytes` from shared `src` to global `dst` (one bulk group).
__device__ __forceinline__ void tma_store(void *dst, const void *src, uint32_t bytes, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
        "r"(smem_u32(src)), "r"(bytes), "l"(pol)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Tile t of the stream: its global start, its length and the position of its
// first element in I ++ J.
struct TmaTile {
    int64_t e0;          // first element within its half
    int len;             // elements, a multiple of 4
    bool hi;             // destination half
};

__device__ __forceinline__ TmaTile tma_tile(int64_t t, int64_t tiles_half, int64_t q4)
{
    TmaTile r;
    r.hi = t >= tiles_half;
    const int64_t tt = r.hi ? t - tiles_half : t;
    r.e0 = tt * kTmaTile;
    const int64_t left = q4 - r.e0;
    r.len = (int)(left < kTmaTile ? left : kTmaTile);
    return r;
}

// RELABEL = false: key[v] = min(key[v], position) for every endpoint (the
// filtering read, then AtomicMin).  RELABEL = true: src_out / dst_out =
// label of every endpoint.
template <bool RELABEL>
__global__ void __launch_bounds__(kTmaBlock) k_lookup_tma(const int32_t *src, const int32_t *dst,
                                                          int64_t m, uint32_t n, uint32_t *key,
                                                          const int32_t *__restrict__ label,
                                                          int32_t *src_out, int32_t *dst_out,
                                                          uint32_t *status)
{
    extern __shared__ __align__(128) int32_t s_buf[];
    __shared__ __align__(8) uint64_t s_bar[kTmaBufs];
    __shared__ int s_fail;
    const int64_t q4 = (m >> 2) << 2;
    const int64_t tiles_half = cdiv(q4, kTmaTile);
    const int64_t tiles = 2 * tiles_half;
    const int64_t G = gridDim.x;
    uint64_t pol = 0;
    if (threadIdx.x == 0) {
        pol = evict_first_policy();
        for (int b = 0; b < kTmaBufs; ++b) mbar_init(&s_bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_fail = 0;
        for (int b = 0; b < kTmaBufs; ++b) {
            const int64_t t = blockIdx.x + (int64_t)b * G;
            if (t >= tiles) break;
            const TmaTile T = tma_tile(t, tiles_half, q4);
            tma_load(s_buf + b * kTmaTile, (T.hi ? dst : src) + T.e0, (uint32_t)T.len * 4u,
                     &s_bar[b], pol);
        }
    }
    __syncthreads();
    int64_t k = 0;
    for (;; ++k) {
        const int64_t t = blockIdx.x + k * G;
        if (t >= tiles) break;
        const int b = (int)(k % kTmaBufs);
        const uint32_t parity = (uint32_t)((k / kTmaBufs) & 1);
        if (!mbar_wait(&s_bar[b], parity)) {
            if (threadIdx.x == 0) raise_status(status, BOBA_ERR_TIMEOUT);
            s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        const TmaTile T = tma_tile(t, tiles_half, q4);
        int4 *buf4 = reinterpret_cast<int4 *>(s_buf + b * kTmaTile);
        constexpr int G4 = kTmaTile / 4 / kTmaBlock;       // int4 groups per thread
        int4 q[G4];
#pragma unroll
        for (int g = 0; g < G4; ++g) {
            const int i4 = g * kTmaBlock + threadIdx.x;
            q[g] = 4 * i4 < T.len ? buf4[i4] : make_int4(0, 0, 0, 0);
        }
        if constexpr (RELABEL) {
            int4 r[G4];
#pragma unroll
            for (int g = 0; g < G4; ++g) {
                const int i4 = g * kTmaBlock + threadIdx.x;
                int32_t *rr = &r[g].x;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t v = comp(q[g], j);
                    rr[j] = -1;
                    if (4 * i4 < T.len) {
                        if ((uint32_t)v < n) rr[j] = __ldg(label + v);
                        else raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < G4; ++g) {
                const int i4 = g * kTmaBlock + threadIdx.x;
                if (4 * i4 < T.len) buf4[i4] = r[g];
            }
            // the labels written by every thread become visible to the bulk copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                tma_store((T.hi ? dst_out : src_out) + T.e0, s_buf + b * kTmaTile,
                          (uint32_t)T.len * 4u, pol);
                // refill the buffer of the previous tile once its store has read it
                if (k >= 1) {
                    const int64_t tn = blockIdx.x + (k - 1 + kTmaBufs) * G;
                    if (tn < tiles) {
                        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                        const int bp = (int)((k - 1) % kTmaBufs);
                        const TmaTile N = tma_tile(tn, tiles_half, q4);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        tma_load(s_buf + bp * kTmaTile, (N.hi ? dst : src) + N.e0,
                                 (uint32_t)N.len * 4u, &s_bar[bp], pol);
                    }
                }
            }
        } else {
            const uint32_t p0 = (uint32_t)((T.hi ? m : 0) + T.e0);
            uint32_t cur[G4][4];
#pragma unroll
            for (int g = 0; g < G4; ++g)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t v = comp(q[g], j);
                    const int i4 = g * kTmaBlock + threadIdx.x;
                    cur[g][j] = (4 * i4 < T.len && (uint32_t)v < n) ? key[v] : 0u;
                }
#pragma unroll
            for (int g = 0; g < G4; ++g) {
                const int i4 = g * kTmaBlock + threadIdx.x;
                if (4 * i4 >= T.len) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t v = comp(q[g], j);
                    if ((uint32_t)v >= n) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                    else first_update(v, p0 + 4u * (uint32_t)i4 + (uint32_t)j, cur[g][j], key);
                }
            }
            __syncthreads();                      // every thread has read buffer b
            if (threadIdx.x == 0) {
                const int64_t tn = blockIdx.x + (k + kTmaBufs) * G;
                if (tn < tiles) {
                    const TmaTile N = tma_tile(tn, tiles_half, q4);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_load(s_buf + b * kTmaTile, (N.hi ? dst : src) + N.e0,
                             (uint32_t)N.len * 4u, &s_bar[b], pol);
                }
            }
        }
    }
    if (s_fail && threadIdx.x == 0) {
        // give the loads already issued the chance to land before the shared
        // memory is released (each wait bounded again)
        for (int64_t j = k; j < k + kTmaBufs; ++j) {
            const int64_t t = blockIdx.x + j * G;
            if (t >= tiles) break;
            (void)mbar_wait(&s_bar[(int)(j % kTmaBufs)], (uint32_t)((j / kTmaBufs) & 1));
        }
    }
    if constexpr (RELABEL) {
        if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    // the up to 3 elements of each half beyond whole quads
    if (blockIdx.x == 0) {
        const int rem = (int)(m - q4);
        if ((int)threadIdx.x < 2 * rem) {
            const bool hi = (int)threadIdx.x >= rem;
            const int64_t e = q4 + (hi ? (int)threadIdx.x - rem : (int)threadIdx.x);
            const int32_t v = (hi ? dst : src)[e];
            if constexpr (RELABEL) {
                int32_t r = -1;
                if ((uint32_t)v < n) r = __ldg(label + v);
                else raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                (hi ? dst_out : src_out)[e] = r;
            } else {
                const uint32_t pos = (uint32_t)((hi ? m : 0) + e);
                if ((uint32_t)v >= n) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                else first_update(v, pos, key[v], key);
            }
        }
    }
}

template <bool RELABEL>
int tma_grid(int64_t m)
{
    static int attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_set[dev & 63]) {
        cudaFuncSetAttribute((const void *)k_lookup_tma<RELABEL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
        attr_set[dev & 63] = 1;
    }
    const int64_t tiles = 2 * cdiv(((m >> 2) << 2), kTmaTile);
    return persistent_grid((const void *)k_lookup_tma<RELABEL>, kTmaBlock, tiles > 0 ? tiles : 1,
                           kTmaSmem);
}

}  // namespace

void launch_first_tma(const ReorderArgs &a, cudaStream_t stream)
{
    const int g = tma_grid<false>(a.m);
    BOBA_TIMED("reorder.first", stream,
               k_lookup_tma<false><<<g, kTmaBlock, kTmaSmem, stream>>>(
                   a.src, a.dst, a.m, a.n, a.key, nullptr, nullptr, nullptr, a.status));
}

void launch_relabel_tma(const ReorderArgs &a, cudaStream_t stream)
{
    const int g = tma_grid<true>(a.m);
    BOBA_TIMED("reorder.relabel", stream,
               k_lookup_tma<true><<<g, kTmaBlock, kTmaSmem, stream>>>(
                   a.src, a.dst, a.m, a.n, nullptr, a.label, a.src_out, a.dst_out, a.status));
}

}  // namespace boba
