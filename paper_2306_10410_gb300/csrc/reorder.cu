// BOBA reordering of one COO graph (arXiv 2306.10410, Sec. 4.3 and Sec. 4.4).
//
// Pipeline (all on one stream, no host synchronisation):
//   k_init      key[v] = SENT; clear the rank bitmap and scan state
//   k_first     key[v] = min position of v in I ++ J           (Alg. 2, AtomicMin)
//   k_mark      bitmap bit key[v] := 1 for every vertex on an edge
//   k_scan      exclusive popcount prefix of the bitmap, one word per 8 bitmap
//               words, single pass with decoupled look-back
//   k_emit      label[v] = rank of key[v] among finite keys, or, for a vertex on
//               no edge, (#vertices on edges) + its rank among such vertices in
//               ascending ID; perm[label[v]] = v                 (ParMapKeys)
//   k_relabel   src_out[e] = label[src[e]], dst_out[e] = label[dst[e]]
//
// The ranks come from the bitmap of first-occurrence positions: bit i is set
// iff position i of I ++ J is the first occurrence of its vertex, which is the
// flag key[I[i]] == i of the method, built from the n keys instead of a second
// pass over the 2m positions.
#include <cstdio>

#include "common.cuh"
#include "host.hpp"
#include "reorder_kernels.cuh"

namespace boba {

// ---------------------------------------------------------------------------
// k_init: key[v] = SENT (Alg. 2's r = infinity^n); zero the bitmap, the
// look-back state and the counters (one contiguous region of the workspace).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_init(uint32_t *__restrict__ key, int64_t n4,
                                              uint32_t *__restrict__ zero, int64_t nzero)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 sent = make_uint4(kSent, kSent, kSent, kSent);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    uint4 *k4 = reinterpret_cast<uint4 *>(key);
    uint4 *z4 = reinterpret_cast<uint4 *>(zero);
    for (int64_t i = t0; i < n4 / 4; i += stride) k4[i] = sent;
    for (int64_t i = t0; i < nzero / 4; i += stride) z4[i] = z;
}

// ---------------------------------------------------------------------------
// k_first: for every position i of I ++ J, key[(I++J)[i]] = min(key, i).
// Alg. 2 (Sec. 4.4) with its update made an AtomicMin, which the paper notes
// yields exactly the lowest position (the order of Alg. 1).
// Work order: the grid sweeps the stream from position 0 upwards in chunks of
// kFirstBlock*kFirstUnroll int4 loads per block, so by the time a position is
// read most earlier positions are already recorded and the filtering read
// (key[v] <= i) skips the atomic.
// ---------------------------------------------------------------------------
// With AGG the lanes of a warp first group equal IDs of the same slot of their
// int4 rounds (__match_any_sync); only the lowest lane of a group, which holds
// the group's lowest position, reads and updates the key (warp-aggregated
// AtomicMin).  The result is the same: the other positions are higher.
template <bool VEC, int BLOCK, int U, bool ATOMIC = true, bool AGG = false>
__device__ __forceinline__ void first_body(const int32_t *__restrict__ src,
                                                       const int32_t *__restrict__ dst, int64_t m,
                                                       uint32_t n, uint32_t *key, uint32_t *status,
                                                       int64_t pos_src, int64_t pos_dst)
{
    const int64_t Q = VEC ? (m >> 2) : 0;   // full int4 quads per half
    if (VEC) {
        const int64_t total = 2 * Q;
        const int64_t chunk = (int64_t)BLOCK * U;
        const int64_t step = (int64_t)gridDim.x * chunk;
        for (int64_t base = (int64_t)blockIdx.x * chunk; base < total; base += step) {
            int4 q[U];
            uint32_t p0[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * BLOCK + threadIdx.x;
                ok[u] = g < total;
                if (ok[u]) {
                    const bool hi = g >= Q;
                    const int64_t qi = hi ? g - Q : g;
                    q[u] = ld_stream(reinterpret_cast<const int4 *>(hi ? dst : src) + qi);
                    p0[u] = (uint32_t)((hi ? pos_dst : pos_src) + 4 * qi);
                } else {
                    q[u] = make_int4(0, 0, 0, 0);
                    p0[u] = 0;
                }
            }
            uint32_t cur[U][4];
            bool lead[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t v = comp(q[u], j);
                    const bool valid = ok[u] && (uint32_t)v < n;
                    lead[u][j] = true;
                    if constexpr (AGG) {
                        // IDs are < 2^31; an invalid slot gets a value of its own
                        const uint32_t tag = valid ? (uint32_t)v : (0x80000000u | (threadIdx.x & 31));
                        const unsigned grp = __match_any_sync(kFull, tag);
                        lead[u][j] = (__ffs(grp) - 1) == (int)(threadIdx.x & 31);
                    }
                    cur[u][j] = (valid && lead[u][j]) ? key[v] : 0u;
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t v = comp(q[u], j);
                    if ((uint32_t)v >= n) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                    else if (lead[u][j]) first_update<ATOMIC>(v, p0[u] + (uint32_t)j, cur[u][j], key);
                }
            }
        }
    }
    // elements not covered by whole quads (all of them when !VEC)
    const int64_t rem = m - 4 * Q;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * rem; t += stride) {
        const bool hi = t >= rem;
        const int64_t e = 4 * Q + (hi ? t - rem : t);
        const int32_t v = ld_stream((hi ? dst : src) + e);
        const uint32_t pos = (uint32_t)((hi ? pos_dst : pos_src) + e);
        if ((uint32_t)v >= n) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
        else first_update<ATOMIC>(v, pos, key[v], key);
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kFirstBlock) k_first(const int32_t *__restrict__ src,
                                                       const int32_t *__restrict__ dst, int64_t m,
                                                       uint32_t n, uint32_t *key, uint32_t *status)
{
    first_body<VEC, kFirstBlock, kFirstUnroll>(src, dst, m, n, key, status, 0, m);
}

// Positions from explicit bases: local edge e holds positions pos_src + e and
// pos_dst + e of the global I ++ J (a shard of a larger graph).
template <bool VEC>
__global__ void __launch_bounds__(kFirstBlock) k_first_at(const int32_t *__restrict__ src,
                                                          const int32_t *__restrict__ dst, int64_t m,
                                                          uint32_t n, uint32_t *key, uint32_t *status,
                                                          int64_t pos_src, int64_t pos_dst)
{
    first_body<VEC, kFirstBlock, kFirstUnroll>(src, dst, m, n, key, status, pos_src, pos_dst);
}

// Alg. 2 exactly as printed (Sec. 4.4): the same sweep with a plain store in
// place of the AtomicMin.  Faster under contention, not deterministic.
template <bool VEC>
__global__ void __launch_bounds__(kFirstBlock) k_first_racy(const int32_t *__restrict__ src,
                                                            const int32_t *__restrict__ dst, int64_t m,
                                                            uint32_t n, uint32_t *key, uint32_t *status)
{
    first_body<VEC, kFirstBlock, kFirstUnroll, false>(src, dst, m, n, key, status, 0, m);
}

// The interleaved flattening drawn in Fig. 1: I(0) J(0) I(1) J(1) ..., edge e's
// source at position 2e and its destination at 2e + 1.
__global__ void __launch_bounds__(256) k_first_interleaved(const int32_t *__restrict__ src,
                                                           const int32_t *__restrict__ dst,
                                                           int64_t m, uint32_t n, uint32_t *key,
                                                           uint32_t *status)
{
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * U;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x) * U + threadIdx.x; b < m; b += stride) {
        int32_t vs[U], vd[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = b + (int64_t)u * blockDim.x;
            vs[u] = vd[u] = -1;
            if (e < m) {
                vs[u] = ld_stream(src + e);
                vd[u] = ld_stream(dst + e);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = b + (int64_t)u * blockDim.x;
            if (e >= m) continue;
            const uint32_t p = (uint32_t)(2 * e);
            if ((uint32_t)vs[u] < n) first_update(vs[u], p, key[vs[u]], key);
            else raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
            if ((uint32_t)vd[u] < n) first_update(vd[u], p + 1, key[vd[u]], key);
            else raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
        }
    }
}

// Variants for the autotuner (vector path): BLOCK threads, U int4 loads in flight.
template <int BLOCK, int U, bool AGG = false>
__global__ void __launch_bounds__(BLOCK) k_first_v(const int32_t *__restrict__ src,
                                                   const int32_t *__restrict__ dst, int64_t m,
                                                   uint32_t n, uint32_t *key, uint32_t *status)
{
    first_body<true, BLOCK, U, true, AGG>(src, dst, m, n, key, status, 0, m);
}

// ---------------------------------------------------------------------------
// k_mark: set bit key[v] of the first-occurrence bitmap for each vertex on an
// edge.  Keys are distinct positions, so bits never collide; words do, hence
// the atomic OR.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mark(const uint32_t *__restrict__ key, int64_t n4,
                                              uint32_t *bitmap)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint4 *k4 = reinterpret_cast<const uint4 *>(key);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4 / 4; i += stride) {
        const uint4 k = k4[i];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (kk[j] != kSent) atomicOr(&bitmap[kk[j] >> 5], 1u << (kk[j] & 31u));
    }
}

// ---------------------------------------------------------------------------
// k_scan: exclusive prefix of the bitmap popcounts, one value per 8 words,
// single pass with decoupled look-back.  The last tile stores the total, the
// number of vertices that lie on an edge.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanBlock) k_scan(const uint32_t *__restrict__ bitmap,
                                                     uint32_t *__restrict__ grp, uint64_t *tstat,
                                                     uint32_t *counters, int64_t tiles,
                                                     uint32_t *status)
{
    __shared__ typename BlockScan<kScanBlock>::Smem sm;
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    __shared__ uint32_t s_rowtot[kScanRows];
    if (threadIdx.x == 0) s_tile = atomicAdd(&counters[kCtrScanTicket], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    // row q of the tile: words tile*T + q*8*kScanBlock .., thread t's sector at 8t
    constexpr int64_t kRowWords = 8 * (int64_t)kScanBlock;
    uint32_t within[kScanRows];
#pragma unroll
    for (int q = 0; q < kScanRows; ++q) {
        const uint4 *w = reinterpret_cast<const uint4 *>(bitmap + tile * kScanTileWords +
                                                         q * kRowWords) + 2 * threadIdx.x;
        const uint4 a = w[0], b = w[1];
        const uint32_t c = __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w) + __popc(b.x) +
                           __popc(b.y) + __popc(b.z) + __popc(b.w);
        uint32_t rt;
        within[q] = BlockScan<kScanBlock>::exclusive(c, &rt, sm);
        if (threadIdx.x == 0) s_rowtot[q] = rt;
        __syncthreads();                   // the scan's shared words are reused
    }
    uint32_t row_before[kScanRows], tot = 0;
#pragma unroll
    for (int q = 0; q < kScanRows; ++q) {
        row_before[q] = tot + within[q];
        tot += s_rowtot[q];
    }
    if (threadIdx.x < 32) {
        const uint64_t p = lookback_exclusive(tstat, tile, tot, status);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScanRows; ++q)
        grp[(tile * kScanTileWords + q * kRowWords) / 8 + threadIdx.x] =
            (uint32_t)(s_prefix + row_before[q]);
    if (tile == tiles - 1 && threadIdx.x == 0) counters[kCtrTotal] = (uint32_t)(s_prefix + tot);
}


// ---------------------------------------------------------------------------
// k_emit: ParMapKeys (Alg. 2): label[v] = rank of key[v]; a vertex on no edge
// gets (#vertices on edges) + its rank among such vertices in ascending ID
// (a look-back scan over vertex tiles); perm[label[v]] = v.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEmitBlock) k_emit(const uint32_t *__restrict__ key, uint32_t n,
                                                     const uint32_t *__restrict__ bitmap,
                                                     const uint32_t *__restrict__ grp,
                                                     int32_t *__restrict__ label,
                                                     int32_t *__restrict__ perm, uint64_t *tstat,
                                                     uint32_t *counters, bool label_vec,
                                                     uint32_t *status)
{
    __shared__ typename BlockScan<kEmitBlock>::Smem sm;
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(&counters[kCtrEmitTicket], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    // row q of the tile is vertices tile*T + q*4*kEmitBlock .. + 4*kEmitBlock - 1
    // and thread t holds its vertices 4t .. 4t+3: the int4 key loads of a row
    // are coalesced, and vertex order is row-major, thread order in a row
    const int64_t v0 = tile * kEmitTileVerts + 4 * (int64_t)threadIdx.x;
    constexpr int64_t kRow = 4 * (int64_t)kEmitBlock;
    uint32_t kk[kEmitGroups][4], cq[kEmitGroups];
#pragma unroll
    for (int q = 0; q < kEmitGroups; ++q) {
        const int64_t vq = v0 + q * kRow;
        uint4 k4 = make_uint4(kSent, kSent, kSent, kSent);
        if (vq < (int64_t)n) k4 = *reinterpret_cast<const uint4 *>(key + vq);   // key padded to 4
        kk[q][0] = k4.x;
        kk[q][1] = k4.y;
        kk[q][2] = k4.z;
        kk[q][3] = k4.w;
        cq[q] = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) cq[q] += (vq + j < (int64_t)n && kk[q][j] == kSent) ? 1u : 0u;
    }
    // vertices on no edge: offset of each row piece inside the tile
    __shared__ uint32_t s_rowtot[kEmitGroups];
    uint32_t within[kEmitGroups];
#pragma unroll
    for (int q = 0; q < kEmitGroups; ++q) {
        uint32_t rt;
        within[q] = BlockScan<kEmitBlock>::exclusive(cq[q], &rt, sm);
        if (threadIdx.x == 0) s_rowtot[q] = rt;
        __syncthreads();                   // the scan's shared words are reused
    }
    uint32_t row_before[kEmitGroups], tot = 0;
#pragma unroll
    for (int q = 0; q < kEmitGroups; ++q) {
        row_before[q] = tot + within[q];
        tot += s_rowtot[q];
    }
    if (threadIdx.x < 32) {
        const uint64_t p = lookback_exclusive(tstat, tile, tot, status);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    const uint32_t on_edges = counters[kCtrTotal];
#pragma unroll
    for (int q = 0; q < kEmitGroups; ++q) {
        const int64_t vq = v0 + q * kRow;
        uint32_t next_iso = on_edges + (uint32_t)s_prefix + row_before[q];
        int32_t lab[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (vq + j >= (int64_t)n) { lab[j] = -1; continue; }
            if (kk[q][j] == kSent) lab[j] = (int32_t)(next_iso++);
            else lab[j] = (int32_t)rank_of_key(kk[q][j], bitmap, grp);
            if ((uint32_t)lab[j] < n) perm[lab[j]] = (int32_t)(vq + j);
            else raise_status(status, BOBA_ERR_TIMEOUT);   // only after a failed look-back
        }
        if (label_vec && vq + 3 < (int64_t)n) {
            *reinterpret_cast<int4 *>(label + vq) = make_int4(lab[0], lab[1], lab[2], lab[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (vq + j < (int64_t)n) label[vq + j] = lab[j];
        }
    }
}

// ---------------------------------------------------------------------------
// k_relabel: rewrite every edge through the labels (Sec. 5.3), edge order
// kept.  src_out/dst_out may alias src/dst: each element is read before the
// same thread writes it.
// ---------------------------------------------------------------------------
// With AGG the lanes of a warp group equal IDs of the same slot of their int4
// rounds; the lowest lane of a group gathers the label and shuffles it to the
// others.
template <bool VEC, int BLOCK, int U, bool AGG = false>
__device__ __forceinline__ void relabel_body(const int32_t *src, const int32_t *dst,
                                                           int64_t m, uint32_t n,
                                                           const int32_t *__restrict__ label,
                                                           int32_t *src_out, int32_t *dst_out,
                                                           uint32_t *status)
{
    const int64_t Q = VEC ? (m >> 2) : 0;
    if (VEC) {
        const int64_t total = 2 * Q;
        const int64_t chunk = (int64_t)BLOCK * U;
        const int64_t step = (int64_t)gridDim.x * chunk;
        for (int64_t base = (int64_t)blockIdx.x * chunk; base < total; base += step) {
            int4 q[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * BLOCK + threadIdx.x;
                if (g < total) {
                    const bool hi = g >= Q;
                    q[u] = ld_stream(reinterpret_cast<const int4 *>(hi ? dst : src) + (hi ? g - Q : g));
                } else if constexpr (AGG) {
                    q[u] = make_int4(0, 0, 0, 0);      // read by the match, never used
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * BLOCK + threadIdx.x;
                if constexpr (AGG) {
                    // every lane takes part in the match and the shuffle
                    int4 r;
                    int32_t *rr = &r.x;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int32_t v = comp(q[u], j);
                        const bool valid = g < total && (uint32_t)v < n;
                        const uint32_t tag = valid ? (uint32_t)v : (0x80000000u | (threadIdx.x & 31));
                        const unsigned grp = __match_any_sync(kFull, tag);
                        const int leader = __ffs(grp) - 1;
                        int32_t x = -1;
                        if (valid && leader == (int)(threadIdx.x & 31)) x = __ldg(label + v);
                        x = __shfl_sync(kFull, x, leader);
                        rr[j] = valid ? x : -1;
                        if (g < total && !valid) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
                    }
                    if (g < total) q[u] = r;
                } else if (g < total) {
                    int4 r;
                    int32_t *rr = &r.x;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int32_t v = comp(q[u], j);
                        if ((uint32_t)v < n) rr[j] = __ldg(label + v);
                        else { rr[j] = -1; raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE); }
                    }
                    q[u] = r;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * BLOCK + threadIdx.x;
                if (g < total) {
                    const bool hi = g >= Q;
                    st_stream(reinterpret_cast<int4 *>(hi ? dst_out : src_out) + (hi ? g - Q : g), q[u]);
                }
            }
        }
    }
    const int64_t rem = m - 4 * Q;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * rem; t += stride) {
        const bool hi = t >= rem;
        const int64_t e = 4 * Q + (hi ? t - rem : t);
        const int32_t v = (hi ? dst : src)[e];
        int32_t r;
        if ((uint32_t)v < n) r = __ldg(label + v);
        else { r = -1; raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE); }
        (hi ? dst_out : src_out)[e] = r;
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kRelabelBlock) k_relabel(const int32_t *src, const int32_t *dst,
                                                           int64_t m, uint32_t n,
                                                           const int32_t *__restrict__ label,
                                                           int32_t *src_out, int32_t *dst_out,
                                                           uint32_t *status)
{
    relabel_body<VEC, kRelabelBlock, kRelabelUnroll>(src, dst, m, n, label, src_out, dst_out, status);
}

template <int BLOCK, int U, bool AGG = false>
__global__ void __launch_bounds__(BLOCK) k_relabel_v(const int32_t *src, const int32_t *dst,
                                                     int64_t m, uint32_t n,
                                                     const int32_t *__restrict__ label,
                                                     int32_t *src_out, int32_t *dst_out,
                                                     uint32_t *status)
{
    relabel_body<true, BLOCK, U, AGG>(src, dst, m, n, label, src_out, dst_out, status);
}

// Launch one tuned variant of the vector-path first-occurrence / relabel kernel.
template <int BLOCK, int U, bool AGG = false>
void launch_first_v(const ReorderArgs &a, cudaStream_t stream)
{
    const int64_t work = cdiv(2 * a.m, 4LL * BLOCK * U);
    const int g = persistent_grid((const void *)k_first_v<BLOCK, U, AGG>, BLOCK, work);
    BOBA_TIMED("reorder.first", stream,
               k_first_v<BLOCK, U, AGG><<<g, BLOCK, 0, stream>>>(a.src, a.dst, a.m, a.n, a.key,
                                                                a.status));
}

template <int BLOCK, int U, bool AGG = false>
void launch_relabel_v(const ReorderArgs &a, cudaStream_t stream)
{
    const int64_t work = cdiv(2 * a.m, 4LL * BLOCK * U);
    const int g = persistent_grid((const void *)k_relabel_v<BLOCK, U, AGG>, BLOCK, work);
    BOBA_TIMED("reorder.relabel", stream,
               k_relabel_v<BLOCK, U, AGG><<<g, BLOCK, 0, stream>>>(a.src, a.dst, a.m, a.n, a.label,
                                                                  a.src_out, a.dst_out, a.status));
}

// Variant table: index -> (block, loads in flight); 6 is the warp-aggregated
// form of the default shape, 7 the form whose edge streams move by bulk
// asynchronous copies (reorder_tma.cu).  Index 0 is the default.
bool launch_first_variant(int v, const ReorderArgs &a, cudaStream_t s)
{
    switch (v) {
    case 1: launch_first_v<256, 2>(a, s); return true;
    case 2: launch_first_v<256, 8>(a, s); return true;
    case 3: launch_first_v<512, 4>(a, s); return true;
    case 4: launch_first_v<128, 8>(a, s); return true;
    case 5: launch_first_v<512, 2>(a, s); return true;
    case 6: launch_first_v<256, 4, true>(a, s); return true;
    case 7: launch_first_tma(a, s); return true;
    default: return false;
    }
}

bool launch_relabel_variant(int v, const ReorderArgs &a, cudaStream_t s)
{
    switch (v) {
    case 1: launch_relabel_v<256, 2>(a, s); return true;
    case 2: launch_relabel_v<256, 8>(a, s); return true;
    case 3: launch_relabel_v<512, 4>(a, s); return true;
    case 4: launch_relabel_v<128, 8>(a, s); return true;
    case 5: launch_relabel_v<512, 2>(a, s); return true;
    case 6: launch_relabel_v<256, 4, true>(a, s); return true;
    case 7: launch_relabel_tma(a, s); return true;
    default: return false;
    }
}

template __global__ void k_first<true>(const int32_t *__restrict__, const int32_t *__restrict__,
                                       int64_t, uint32_t, uint32_t *, uint32_t *);
template __global__ void k_first<false>(const int32_t *__restrict__, const int32_t *__restrict__,
                                        int64_t, uint32_t, uint32_t *, uint32_t *);
template __global__ void k_first_at<true>(const int32_t *__restrict__, const int32_t *__restrict__,
                                          int64_t, uint32_t, uint32_t *, uint32_t *, int64_t,
                                          int64_t);
template __global__ void k_relabel<true>(const int32_t *, const int32_t *, int64_t, uint32_t,
                                         const int32_t *__restrict__, int32_t *, int32_t *,
                                         uint32_t *);
template __global__ void k_relabel<false>(const int32_t *, const int32_t *, int64_t, uint32_t,
                                          const int32_t *__restrict__, int32_t *, int32_t *,
                                          uint32_t *);

boba_status_t launch_reorder(const ReorderArgs &a, int64_t n4, size_t nzero_u32,
                             cudaStream_t stream)
{
    {
        const int64_t work = cdiv((int64_t)((size_t)n4 > nzero_u32 ? (size_t)n4 : nzero_u32) / 4, 256);
        const int g = persistent_grid((const void *)k_init, 256, work);
        BOBA_TIMED("reorder.init", stream,
                   k_init<<<g, 256, 0, stream>>>(a.key, n4, a.bitmap, (int64_t)nzero_u32));
    }
    if (a.m > 0 && a.variant != 0) {
        const bool vec = aligned16(a.src) && aligned16(a.dst);
        const int64_t work = cdiv(2 * a.m, 4 * kFirstBlock * kFirstUnroll);
        if (a.variant == 1) {
            const int g = persistent_grid((const void *)k_first_interleaved, 256, cdiv(a.m, 1024));
            BOBA_TIMED("reorder.first", stream,
                       k_first_interleaved<<<g, 256, 0, stream>>>(a.src, a.dst, a.m, a.n, a.key, a.status));
        } else if (vec) {
            const int g = persistent_grid((const void *)k_first_racy<true>, kFirstBlock, work);
            BOBA_TIMED("reorder.first", stream,
                       k_first_racy<true><<<g, kFirstBlock, 0, stream>>>(a.src, a.dst, a.m, a.n, a.key,
                                                                        a.status));
        } else {
            const int g = persistent_grid((const void *)k_first_racy<false>, kFirstBlock, work * 4);
            BOBA_TIMED("reorder.first", stream,
                       k_first_racy<false><<<g, kFirstBlock, 0, stream>>>(a.src, a.dst, a.m, a.n,
                                                                         a.key, a.status));
        }
    } else if (a.m > 0) {
        const bool vec = aligned16(a.src) && aligned16(a.dst);
        const int64_t work = cdiv(2 * a.m, 4 * kFirstBlock * kFirstUnroll);
        if (vec && launch_first_variant(tuned_variant(kTuneFirst, a.m), a, stream)) {
            // tuned variant launched
        } else if (vec) {
            const int g = persistent_grid((const void *)k_first<true>, kFirstBlock, work);
            BOBA_TIMED("reorder.first", stream,
                       k_first<true><<<g, kFirstBlock, 0, stream>>>(a.src, a.dst, a.m, a.n, a.key,
                                                                   a.status));
        } else {
            const int g = persistent_grid((const void *)k_first<false>, kFirstBlock, work * 4);
            BOBA_TIMED("reorder.first", stream,
                       k_first<false><<<g, kFirstBlock, 0, stream>>>(a.src, a.dst, a.m, a.n, a.key,
                                                                    a.status));
        }
    }
    if (a.m > 0) {
        const int gm = persistent_grid((const void *)k_mark, 256, cdiv(n4 / 4, 256));
        BOBA_TIMED("reorder.mark", stream, k_mark<<<gm, 256, 0, stream>>>(a.key, n4, a.bitmap));
        BOBA_TIMED("reorder.scan", stream,
                   k_scan<<<(unsigned)a.scan_tiles, kScanBlock, 0, stream>>>(
                       a.bitmap, a.grp, a.tstat_scan, a.counters, a.scan_tiles, a.status));
    }
    BOBA_TIMED("reorder.emit", stream,
               k_emit<<<(unsigned)a.emit_tiles, kEmitBlock, 0, stream>>>(
                   a.key, a.n, a.bitmap, a.grp, a.label, a.perm, a.tstat_emit, a.counters,
                   a.label_vec, a.status));
    if (a.src_out && a.m > 0) {
        const bool vec = aligned16(a.src) && aligned16(a.dst) && aligned16(a.src_out) &&
                         aligned16(a.dst_out);
        const int64_t work = cdiv(2 * a.m, 4 * kRelabelBlock * kRelabelUnroll);
        if (vec && launch_relabel_variant(tuned_variant(kTuneRelabel, a.m), a, stream)) {
            // tuned variant launched
        } else if (vec) {
            const int g = persistent_grid((const void *)k_relabel<true>, kRelabelBlock, work);
            BOBA_TIMED("reorder.relabel", stream,
                       k_relabel<true><<<g, kRelabelBlock, 0, stream>>>(
                           a.src, a.dst, a.m, a.n, a.label, a.src_out, a.dst_out, a.status));
        } else {
            const int g = persistent_grid((const void *)k_relabel<false>, kRelabelBlock, work * 4);
            BOBA_TIMED("reorder.relabel", stream,
                       k_relabel<false><<<g, kRelabelBlock, 0, stream>>>(
                           a.src, a.dst, a.m, a.n, a.label, a.src_out, a.dst_out, a.status));
        }
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

}  // namespace boba

using namespace boba;

extern "C" size_t boba_reorder_workspace_bytes(int64_t m, int64_t n)
{
    ReorderLayout L;
    if (!reorder_layout(m, n, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_reorder_ex(const int32_t *src, const int32_t *dst, int64_t m,
                                         int64_t n, int32_t *perm_out, int32_t *src_out,
                                         int32_t *dst_out, int32_t *label_out, void *ws,
                                         size_t ws_bytes, void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if ((src_out == nullptr) != (dst_out == nullptr)) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (perm_out == nullptr || ws == nullptr) return BOBA_ERR_INVALID_ARG;
    if (m > 0 && (src == nullptr || dst == nullptr)) return BOBA_ERR_INVALID_ARG;
    ReorderLayout L;
    reorder_layout(m, n, L);
    if (ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);

    char *base = static_cast<char *>(ws);
    ReorderArgs a;
    a.src = src;
    a.dst = dst;
    a.m = m;
    a.n = (uint32_t)n;
    a.key = reinterpret_cast<uint32_t *>(base + L.key);
    a.label = label_out ? label_out : reinterpret_cast<int32_t *>(base + L.label);
    a.perm = perm_out;
    a.bitmap = reinterpret_cast<uint32_t *>(base + L.bitmap);
    a.grp = reinterpret_cast<uint32_t *>(base + L.grp);
    a.tstat_scan = reinterpret_cast<uint64_t *>(base + L.tstat_scan);
    a.tstat_emit = reinterpret_cast<uint64_t *>(base + L.tstat_emit);
    a.counters = reinterpret_cast<uint32_t *>(base + L.counters);
    a.nwords = L.nwords;
    a.scan_tiles = L.scan_tiles;
    a.emit_tiles = L.emit_tiles;
    a.status = dev->status;
    a.src_out = src_out;
    a.dst_out = dst_out;
    a.label_vec = aligned16(a.label);
    return launch_reorder(a, L.n4, (L.zero_end - L.zero_begin) / 4, stream);
}

// ---------------------------------------------------------------------------
// The three phases as separate entry points (for sharding a graph over
// several devices: local keys, a MIN merge of the key arrays, then labels and
// relabel on every device).
// ---------------------------------------------------------------------------

extern "C" boba_status_t boba_first_keys(const int32_t *src, const int32_t *dst, int64_t m_local,
                                         int64_t pos_src, int64_t pos_dst, int64_t n,
                                         uint32_t *key, int init, void *stream_)
{
    if (m_local < 0 || n < 0 || pos_src < 0 || pos_dst < 0) return BOBA_ERR_INVALID_ARG;
    if (m_local > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (pos_src + m_local > 2 * kMaxSize || pos_dst + m_local > 2 * kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0) return m_local == 0 ? BOBA_OK : BOBA_ERR_INVALID_ARG;
    if (key == nullptr || (m_local > 0 && (src == nullptr || dst == nullptr))) return BOBA_ERR_INVALID_ARG;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (init) BOBA_CUDA_TRY(cudaMemsetAsync(key, 0xFF, (size_t)n * 4, stream));
    if (m_local > 0) {
        const bool vec = aligned16(src) && aligned16(dst);
        const int64_t work = cdiv(2 * m_local, 4 * kFirstBlock * kFirstUnroll);
        if (vec) {
            const int g = persistent_grid((const void *)k_first_at<true>, kFirstBlock, work);
            BOBA_TIMED("reorder.first", stream,
                       k_first_at<true><<<g, kFirstBlock, 0, stream>>>(src, dst, m_local, (uint32_t)n,
                                                                      key, dev->status, pos_src,
                                                                      pos_dst));
        } else {
            const int g = persistent_grid((const void *)k_first_at<false>, kFirstBlock, work * 4);
            BOBA_TIMED("reorder.first", stream,
                       k_first_at<false><<<g, kFirstBlock, 0, stream>>>(src, dst, m_local,
                                                                       (uint32_t)n, key,
                                                                       dev->status, pos_src,
                                                                       pos_dst));
        }
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

extern "C" size_t boba_labels_workspace_bytes(int64_t m_total, int64_t n)
{
    return boba_reorder_workspace_bytes(m_total, n);
}

extern "C" boba_status_t boba_labels_from_keys(const uint32_t *key, int64_t m_total, int64_t n,
                                               int32_t *perm_out, int32_t *label_out, void *ws,
                                               size_t ws_bytes, void *stream_)
{
    if (m_total < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m_total > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0) return BOBA_OK;
    if (key == nullptr || perm_out == nullptr || ws == nullptr) return BOBA_ERR_INVALID_ARG;
    ReorderLayout L;
    reorder_layout(m_total, n, L);
    if (ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *base = static_cast<char *>(ws);
    uint32_t *kcopy = reinterpret_cast<uint32_t *>(base + L.key);
    // the kernels read keys padded to a multiple of 4 with SENT
    const int64_t nzero = (int64_t)((L.zero_end - L.zero_begin) / 4);
    {
        const int64_t work = cdiv((L.n4 > nzero ? L.n4 : nzero) / 4, 256);
        const int g = persistent_grid((const void *)k_init, 256, work);
        BOBA_TIMED("reorder.init", stream,
                   k_init<<<g, 256, 0, stream>>>(kcopy, L.n4,
                                                 reinterpret_cast<uint32_t *>(base + L.bitmap), nzero));
    }
    BOBA_CUDA_TRY(cudaMemcpyAsync(kcopy, key, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream));
    ReorderArgs a;
    a.src = nullptr;
    a.dst = nullptr;
    a.m = m_total;
    a.n = (uint32_t)n;
    a.key = kcopy;
    a.label = label_out ? label_out : reinterpret_cast<int32_t *>(base + L.label);
    a.perm = perm_out;
    a.bitmap = reinterpret_cast<uint32_t *>(base + L.bitmap);
    a.grp = reinterpret_cast<uint32_t *>(base + L.grp);
    a.tstat_scan = reinterpret_cast<uint64_t *>(base + L.tstat_scan);
    a.tstat_emit = reinterpret_cast<uint64_t *>(base + L.tstat_emit);
    a.counters = reinterpret_cast<uint32_t *>(base + L.counters);
    a.nwords = L.nwords;
    a.scan_tiles = L.scan_tiles;
    a.emit_tiles = L.emit_tiles;
    a.status = dev->status;
    a.src_out = nullptr;
    a.dst_out = nullptr;
    a.label_vec = aligned16(a.label);
    if (m_total > 0) {
        const int gm = persistent_grid((const void *)k_mark, 256, cdiv(L.n4 / 4, 256));
        BOBA_TIMED("reorder.mark", stream, k_mark<<<gm, 256, 0, stream>>>(a.key, L.n4, a.bitmap));
        BOBA_TIMED("reorder.scan", stream,
                   k_scan<<<(unsigned)a.scan_tiles, kScanBlock, 0, stream>>>(
                       a.bitmap, a.grp, a.tstat_scan, a.counters, a.scan_tiles, a.status));
    }
    BOBA_TIMED("reorder.emit", stream,
               k_emit<<<(unsigned)a.emit_tiles, kEmitBlock, 0, stream>>>(
                   a.key, a.n, a.bitmap, a.grp, a.label, a.perm, a.tstat_emit, a.counters,
                   a.label_vec, a.status));
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

extern "C" boba_status_t boba_relabel(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                      const int32_t *label, int32_t *src_out, int32_t *dst_out,
                                      void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (m == 0) return BOBA_OK;
    if (!src || !dst || !label || !src_out || !dst_out) return BOBA_ERR_INVALID_ARG;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    const bool vec = aligned16(src) && aligned16(dst) && aligned16(src_out) && aligned16(dst_out);
    const int64_t work = cdiv(2 * m, 4 * kRelabelBlock * kRelabelUnroll);
    if (vec) {
        const int g = persistent_grid((const void *)k_relabel<true>, kRelabelBlock, work);
        BOBA_TIMED("reorder.relabel", stream,
                   k_relabel<true><<<g, kRelabelBlock, 0, stream>>>(src, dst, m, (uint32_t)n, label,
                                                                   src_out, dst_out, dev->status));
    } else {
        const int g = persistent_grid((const void *)k_relabel<false>, kRelabelBlock, work * 4);
        BOBA_TIMED("reorder.relabel", stream,
                   k_relabel<false><<<g, kRelabelBlock, 0, stream>>>(src, dst, m, (uint32_t)n, label,
                                                                    src_out, dst_out, dev->status));
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

extern "C" boba_status_t boba_reorder_variant(const int32_t *src, const int32_t *dst, int64_t m,
                                              int64_t n, int32_t *perm_out, int32_t *src_out,
                                              int32_t *dst_out, int variant, void *ws,
                                              size_t ws_bytes, void *stream_)
{
    if (variant < 0 || variant > 2) return BOBA_ERR_INVALID_ARG;
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if ((src_out == nullptr) != (dst_out == nullptr)) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (perm_out == nullptr || ws == nullptr) return BOBA_ERR_INVALID_ARG;
    if (m > 0 && (src == nullptr || dst == nullptr)) return BOBA_ERR_INVALID_ARG;
    ReorderLayout L;
    reorder_layout(m, n, L);
    if (ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    char *base = static_cast<char *>(ws);
    ReorderArgs a;
    a.src = src;
    a.dst = dst;
    a.m = m;
    a.n = (uint32_t)n;
    a.key = reinterpret_cast<uint32_t *>(base + L.key);
    a.label = reinterpret_cast<int32_t *>(base + L.label);
    a.perm = perm_out;
    a.bitmap = reinterpret_cast<uint32_t *>(base + L.bitmap);
    a.grp = reinterpret_cast<uint32_t *>(base + L.grp);
    a.tstat_scan = reinterpret_cast<uint64_t *>(base + L.tstat_scan);
    a.tstat_emit = reinterpret_cast<uint64_t *>(base + L.tstat_emit);
    a.counters = reinterpret_cast<uint32_t *>(base + L.counters);
    a.nwords = L.nwords;
    a.scan_tiles = L.scan_tiles;
    a.emit_tiles = L.emit_tiles;
    a.status = dev->status;
    a.src_out = src_out;
    a.dst_out = dst_out;
    a.label_vec = true;
    a.variant = variant;
    return launch_reorder(a, L.n4, (L.zero_end - L.zero_begin) / 4, static_cast<cudaStream_t>(stream_));
}
