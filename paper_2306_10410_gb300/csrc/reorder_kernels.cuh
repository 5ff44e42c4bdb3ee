// Device building blocks of the BOBA reordering, shared by the single-graph
// path and the batched path.
#pragma once

#include "common.cuh"
#include "host.hpp"

namespace boba {

constexpr int kFirstBlock = 256;        // threads per block, first-occurrence pass
constexpr int kFirstUnroll = 4;         // int4 loads in flight per thread
constexpr int kRelabelBlock = 256;
constexpr int kRelabelUnroll = 4;
constexpr int kScanBlock = 256;
constexpr int kScanRows = 4;                        // rows of 8 bitmap words per thread
constexpr int kScanTileWords = kScanBlock * 8 * kScanRows;   // a thread: one 32-byte sector per row
constexpr int kEmitBlock = 256;
constexpr int kEmitGroups = 4;                      // int4 groups of keys per thread
constexpr int kEmitTileVerts = kEmitBlock * 4 * kEmitGroups;   // 16 vertices per thread
constexpr int kNumCounters = 8;                    // tickets and totals in the workspace
constexpr int kCtrScanTicket = 0, kCtrEmitTicket = 1, kCtrTotal = 2;

struct ReorderArgs {
    const int32_t *src, *dst;
    int64_t m;
    uint32_t n;
    uint32_t *key;
    int32_t *label;
    int32_t *perm;
    uint32_t *bitmap;       // nwords words, bit i = position i is a first occurrence
    uint32_t *grp;          // exclusive popcount prefix, one per 8 bitmap words
    uint64_t *tstat_scan, *tstat_emit;
    uint32_t *counters;
    int64_t nwords, scan_tiles, emit_tiles;
    uint32_t *status;
    int32_t *src_out, *dst_out;
    bool label_vec;
    int variant = 0;          // 0 first occurrence in I ++ J, 1 interleaved, 2 racy store
};

// One position of I ++ J: lower key[v] to `pos` unless a position already
// recorded for v is lower.  The filtering read may see a stale value: keys only
// ever decrease, so a stale key is >= the current one and at worst costs an
// atomic that changes nothing; the minimum itself is taken by atomicMin.
template <bool ATOMIC = true>
__device__ __forceinline__ void first_update(int32_t v, uint32_t pos, uint32_t cur, uint32_t *key)
{
    if constexpr (ATOMIC) {
        if (cur > pos) atomicMin(&key[v], pos);
    } else {
        // Alg. 2 exactly as printed: a plain, racy store (the result depends
        // on timing; the minimum is not guaranteed)
        if (cur > pos) key[v] = pos;
    }
}

// Rank of a finite key among all first-occurrence positions: the popcount of
// the bitmap below bit k.  grp[g] holds the count below word 8g; the eight
// words of group g form one aligned 32-byte sector.
__device__ __forceinline__ uint32_t rank_of_key(uint32_t k, const uint32_t *__restrict__ bitmap,
                                                const uint32_t *__restrict__ grp)
{
    const uint32_t g = k >> 8;
    const uint4 *gw = reinterpret_cast<const uint4 *>(bitmap) + 2 * (size_t)g;
    const uint4 a = gw[0], b = gw[1];
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const uint32_t wi = (k >> 5) & 7u;
    uint32_t r = grp[g];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((uint32_t)i < wi) r += __popc(w[i]);
        else if ((uint32_t)i == wi) r += __popc(w[i] & ((1u << (k & 31u)) - 1u));
    }
    return r;
}

__device__ __forceinline__ int32_t comp(const int4 &q, int j)
{
    return j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
}

// Workspace layout of one reorder (byte offsets from a 256-byte-aligned base).
struct ReorderLayout {
    int64_t n4, nwords, ngroups, scan_tiles, emit_tiles;
    size_t key, label, grp, zero_begin, bitmap, tstat_scan, tstat_emit, counters, zero_end, total;
};

inline bool reorder_layout(int64_t m, int64_t n, ReorderLayout &L)
{
    if (m < 0 || n < 0 || m > kMaxSize || n > kMaxSize) return false;
    L.n4 = align_up((size_t)(n > 0 ? n : 1), 4);
    L.nwords = (int64_t)align_up((size_t)cdiv(2 * m, 32) > 0 ? (size_t)cdiv(2 * m, 32) : 1,
                                 kScanTileWords);
    L.ngroups = L.nwords / 8;
    L.scan_tiles = L.nwords / kScanTileWords;
    L.emit_tiles = cdiv(n > 0 ? n : 1, kEmitTileVerts);
    Carve c;
    L.key = c.take(L.n4 * 4);
    L.label = c.take(L.n4 * 4);
    L.grp = c.take(L.ngroups * 4);
    L.zero_begin = c.off;
    L.bitmap = c.take(L.nwords * 4);
    L.tstat_scan = c.take(L.scan_tiles * 8);
    L.tstat_emit = c.take(L.emit_tiles * 8);
    L.counters = c.take(kNumCounters * 4);
    L.zero_end = c.off;
    L.total = c.off;
    return true;
}

boba_status_t launch_reorder(const ReorderArgs &a, int64_t n4, size_t nzero_u32,
                             cudaStream_t stream);

// The lookup passes with their edge streams moved by bulk asynchronous copies
// (reorder_tma.cu); vector path only (16-byte-aligned arrays).
void launch_first_tma(const ReorderArgs &a, cudaStream_t stream);
void launch_relabel_tma(const ReorderArgs &a, cudaStream_t stream);

// The kernels of the pipeline (defined in reorder.cu).
__global__ void k_init(uint32_t *__restrict__ key, int64_t n4, uint32_t *__restrict__ zero,
                       int64_t nzero);
template <bool VEC>
__global__ void k_first(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                        int64_t m, uint32_t n, uint32_t *key, uint32_t *status);
__global__ void k_mark(const uint32_t *__restrict__ key, int64_t n4, uint32_t *bitmap);
__global__ void k_scan(const uint32_t *__restrict__ bitmap, uint32_t *__restrict__ grp,
                       uint64_t *tstat, uint32_t *counters, int64_t tiles, uint32_t *status);
__global__ void k_emit(const uint32_t *__restrict__ key, uint32_t n,
                       const uint32_t *__restrict__ bitmap, const uint32_t *__restrict__ grp,
                       int32_t *__restrict__ label, int32_t *__restrict__ perm, uint64_t *tstat,
                       uint32_t *counters, bool label_vec, uint32_t *status);
template <bool VEC>
__global__ void k_relabel(const int32_t *src, const int32_t *dst, int64_t m, uint32_t n,
                          const int32_t *__restrict__ label, int32_t *src_out, int32_t *dst_out,
                          uint32_t *status);

}  // namespace boba
