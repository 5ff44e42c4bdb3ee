// Batched BOBA: G independent graphs of uneven sizes reordered together
// (arXiv 2306.10410, Alg. 2 with AtomicMin, per graph).  No work crosses a
// graph boundary, so graphs need no coordination with each other.
//
// Two modes (the second is the default; an autotuner can pick either):
//
//  kBatchCluster -- one persistent cluster launch.  A graph with at most kKcap
//     vertices is reordered by a single CTA with its keys, then labels, in that
//     CTA's shared memory; a larger graph (up to kTeam * kKcap vertices) by a
//     cluster of kTeam CTAs whose shared memories hold one slice each of the
//     key/label array, reached through distributed shared memory.  Items are
//     claimed largest first: large graphs, then packs of kTeam small graphs.
//
//  kBatchSplit -- small graphs as above but in a persistent launch without
//     clusters (every SM takes part), and the graphs above kKcap vertices all
//     together, phase by phase, in six grid-wide launches with their keys in
//     global memory: init, first occurrence, mark, bitmap scan, emit,
//     relabel.  Each phase maps a chunk or tile to its graph through
//     per-graph tile counts (resuming from the previous chunk's graph, else a
//     binary search); the two look-back scans are segmented by letting the
//     first tile of each graph publish its prefix at once.  The
//     first-occurrence and relabel phases of graphs of up to a few slices of
//     kKcap vertices can instead run sliced: one CTA per (graph, slice) holds
//     the slice's keys or labels in shared memory and streams all of the
//     graph's endpoints (the schedules of batch_slices).  Measured on GB300,
//     distributed shared memory was slower than L2 for the random key
//     accesses of large graphs, hence this default.
//
// In both modes a graph goes through the steps of the single-graph path: keys =
// SENT, first occurrence, first-occurrence bitmap, popcount prefix, labels
// (rank of the key; vertices on no edge after them by ascending ID), perm, and
// the relabel of both endpoint arrays.  k_batch_plan validates the offsets,
// orders the graphs (large first, each class by decreasing edge count in
// power-of-two buckets) and tabulates the tiles of the large graphs.
#include <cooperative_groups.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "host.hpp"

namespace cg = cooperative_groups;

namespace boba {
namespace {

constexpr int kBB = 1024;                  // threads per CTA of the per-graph kernels
constexpr int kTeam = 8;                   // CTAs per cluster, team size for large graphs
constexpr int kKcap = 54 * 1024;           // vertices per CTA held in shared memory
constexpr size_t kDynSmem = (size_t)kKcap * 4;
constexpr int kU = 8;                      // stream loads in flight per thread
constexpr int64_t kSmallMaxM = 1ll << 21;  // split mode: graphs with more edges go to the phase path
constexpr int kHdrItems = 0, kHdrLarge = 1, kHdrTicket = 2, kHdrValid = 3, kHdrScanTicket = 4,
              kHdrEmitTicket = 5, kHdrSliceFirst = 6, kHdrSliceRelabel = 7, kHdrRunTicket = 8,
              kHdrFirstRunTicket = 9;
constexpr int kMaxSlices = 8;              // sliced large path: n <= kMaxSlices * kKcap

// tiles of the phase-batched large-graph path
constexpr int kLB = 256;                   // threads per block
constexpr int kPosChunk = kLB * 64;        // positions of I ++ J per block step (4 rounds of 16)
constexpr int kBlRows = 4;                 // rows per tile: a thread takes one piece of each
constexpr int kVtxRow = kLB * 4;           // vertices per row (one int4 of keys per thread)
constexpr int kWordRow = kLB * 8;          // bitmap words per row (one 32-byte sector per thread)
constexpr int kVtxTile = kVtxRow * kBlRows;     // vertices per tile
constexpr int kWordTile = kWordRow * kBlRows;   // bitmap words per scan tile
constexpr int kEdgeChunk = kLB * 32;       // edges per relabel block step (4 rounds of 8 per thread)

enum BatchMode { kBatchCluster = 0, kBatchSplit = 1 };

struct BatchArgs {
    const int32_t *src, *dst;
    const int64_t *eoff, *voff;
    int64_t G, max_m, max_n, total_m, total_n;
    int32_t *perm, *so, *dout;
    uint32_t *hdr;           // items, large graphs, ticket, valid graphs, scan/emit tickets
    uint32_t *order;         // graph ids in processing order
    uint32_t *scratch;       // one region per CTA of the per-graph kernel
    int64_t region_words;    // wmax bitmap words + wmax/8 group-prefix words
    int64_t wmax;
    uint32_t *status;
    int large_threshold;     // graphs with more vertices go to the team / phase path
    int64_t small_max_m;     // ... and, in split mode, graphs with more edges
    int64_t n_limit;         // largest graph the mode can take
    // phase-batched large-graph path (prefix tables over the large graphs, L+1 entries)
    uint32_t *lg_pc, *lg_vt, *lg_wt, *lg_ec, *lg_tot, *lg_st;
    uint32_t *kl;            // keys, then labels, of the large graphs (vertex-tile padded)
    uint32_t *lbm;           // bitmaps of the large graphs (word-tile padded)
    uint32_t *lgrp;          // group prefixes (one per 8 words)
    uint64_t *lts_scan, *lts_emit;
    int64_t lts_scan_cap, lts_emit_cap;
    // sliced large path: graphs of at most this many slices take the sliced
    // first-occurrence / relabel kernel, the others the global one (0: none)
    int first_smax, relabel_smax;
    // the global first-occurrence pass / relabel claims runs of consecutive
    // chunks, one CTA per SM (k_bl_first_runs, k_bl_relabel_runs), instead of
    // striding over the chunks
    bool first_runs, relabel_runs;
};

__device__ __forceinline__ int floor_log2_p1(int64_t x)   // floor(log2(x + 1)), x >= 0
{
    return 63 - __clzll((unsigned long long)(x + 1));
}

__device__ __forceinline__ bool graph_ok(const BatchArgs &a, int64_t g, int64_t &m, int64_t &n)
{
    const int64_t e0 = a.eoff[g], e1 = a.eoff[g + 1], v0 = a.voff[g], v1 = a.voff[g + 1];
    m = e1 - e0;
    n = v1 - v0;
    return e0 >= 0 && v0 >= 0 && m >= 0 && n >= 0 && e1 <= a.total_m && v1 <= a.total_n &&
           m <= a.max_m && n <= a.max_n && n <= a.n_limit && !(n == 0 && m > 0);
}

// One block of 1024 threads: validate the offsets, bucket the graphs, write
// the processing order and the work header, reset the tickets, and tabulate
// the tiles of the large graphs (exclusive prefixes over order[0 .. L)).
__global__ void __launch_bounds__(1024) k_batch_plan(BatchArgs a)
{
    __shared__ uint32_t hist[128], cur[128];
    __shared__ typename BlockScan<1024>::Smem sm;
    __shared__ uint32_t carry[5];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t g = threadIdx.x; g < a.G; g += blockDim.x) {
        int64_t m, n;
        if (!graph_ok(a, g, m, n)) { raise_status(a.status, BOBA_ERR_INVALID_ARG); continue; }
        if (n == 0) continue;
        const bool large = n > a.large_threshold || m > a.small_max_m;
        const int b = (large ? 0 : 64) + (63 - (floor_log2_p1(m) & 63));
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0, large = 0;
        for (int b = 0; b < 128; ++b) {
            cur[b] = s;
            s += hist[b];
            if (b < 64) large += hist[b];
        }
        a.hdr[kHdrLarge] = large;
        a.hdr[kHdrValid] = s;
        a.hdr[kHdrItems] = large + (s - large + kTeam - 1) / kTeam;
        a.hdr[kHdrTicket] = 0;
        a.hdr[kHdrScanTicket] = 0;
        a.hdr[kHdrEmitTicket] = 0;
        a.hdr[kHdrSliceFirst] = 0;
        a.hdr[kHdrSliceRelabel] = 0;
        a.hdr[kHdrRunTicket] = 0;
        a.hdr[kHdrFirstRunTicket] = 0;
        for (int k = 0; k < 5; ++k) carry[k] = 0;
    }
    __syncthreads();
    for (int64_t g = threadIdx.x; g < a.G; g += blockDim.x) {
        int64_t m, n;
        if (!graph_ok(a, g, m, n) || n == 0) continue;
        const bool large = n > a.large_threshold || m > a.small_max_m;
        const int b = (large ? 0 : 64) + (63 - (floor_log2_p1(m) & 63));
        a.order[atomicAdd(&cur[b], 1u)] = (uint32_t)g;
    }
    __syncthreads();
    if (a.lg_pc == nullptr) return;
    const uint32_t L = a.hdr[kHdrLarge];
    for (uint32_t base = 0; base <= L; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        uint32_t c[5] = {0, 0, 0, 0, 0};
        if (j < L) {
            const uint32_t g = a.order[j];
            const int64_t m = a.eoff[g + 1] - a.eoff[g], n = a.voff[g + 1] - a.voff[g];
            c[0] = (uint32_t)cdiv(2 * m, kPosChunk);
            c[1] = (uint32_t)cdiv(n, kVtxTile);
            const int64_t words = cdiv(2 * m, 32) > 0 ? cdiv(2 * m, 32) : 1;
            c[2] = (uint32_t)cdiv(words, kWordTile);
            c[3] = (uint32_t)cdiv(m, kEdgeChunk);
            c[4] = (uint32_t)cdiv(n, kKcap);
        }
        uint32_t *tabs[5] = {a.lg_pc, a.lg_vt, a.lg_wt, a.lg_ec, a.lg_st};
        for (int k = 0; k < 5; ++k) {
            uint32_t tot;
            const uint32_t ex = BlockScan<1024>::exclusive(c[k], &tot, sm);
            if (j <= L) tabs[k][j] = carry[k] + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry[k] += tot;
            __syncthreads();
        }
    }
}

struct TeamSmem {
    typename BlockScan<kBB>::Smem scan;
    uint32_t *kp[kTeam];     // key/label array of each team member (generic addresses)
    uint32_t base[kTeam];    // bitmap rank base of each member's word slice
    uint32_t xtot, xiso;     // this CTA's bitmap total and isolated count (read by the team)
    uint32_t on_edges, iso_before;
    uint32_t item;
};

template <int T>
__device__ __forceinline__ void team_sync(cg::cluster_group *cl)
{
    if constexpr (T == 1) __syncthreads();
    else cl->sync();
}

template <int T>
__device__ __forceinline__ uint32_t *key_ptr(uint32_t *s_keys, TeamSmem &ts, uint32_t owner)
{
    if constexpr (T == 1) return s_keys;
    else return ts.kp[owner];
}

// The team member whose bitmap slice of Wc words holds bitmap word w.  One
// CTA alone owns every word; in a team w < 2^27 (keys are 32-bit positions),
// so a 32-bit division suffices.
template <int T>
__device__ __forceinline__ uint32_t owner_of_word(uint32_t w, int64_t Wc)
{
    if constexpr (T == 1) return 0u;
    else return w / (uint32_t)Wc;
}

// Process graph g with a team of T CTAs; this CTA is member t, the team's CTAs
// are grid CTAs cta0 .. cta0+T-1 (their scratch regions).
template <int T>
__device__ void process_graph(const BatchArgs &a, uint32_t g, int t, int64_t cta0,
                              cg::cluster_group *cl, uint32_t *s_keys, TeamSmem &ts)
{
    const int tid = threadIdx.x;
    const int64_t E0 = a.eoff[g], m = a.eoff[g + 1] - E0;
    const int64_t V0 = a.voff[g], n = a.voff[g + 1] - V0;
    const uint32_t nn = (uint32_t)n;
    const uint32_t chunk = (uint32_t)cdiv(n, T);
    const int64_t v_lo = (int64_t)t * chunk;
    const int64_t myn = n - v_lo < 0 ? 0 : (n - v_lo < chunk ? n - v_lo : chunk);
    const int64_t W = (int64_t)align_up((size_t)(cdiv(2 * m, 32) > 0 ? cdiv(2 * m, 32) : 1),
                                        (size_t)8 * T);
    const int64_t Wc = W / T;
    uint32_t *const my_bm = a.scratch + (cta0 + t) * a.region_words;
    uint32_t *const my_grp = my_bm + a.wmax;

    if constexpr (T > 1) {
        if (tid < T) ts.kp[tid] = cl->map_shared_rank(s_keys, tid);
    }
    // 1. keys = SENT, clear this member's bitmap slice
    for (int64_t i = tid; i < myn; i += kBB) s_keys[i] = kSent;
    for (int64_t w = tid; w < Wc; w += kBB) my_bm[w] = 0u;
    team_sync<T>(cl);

    // 2. first occurrence over this member's share of I ++ J: kU loads in
    // flight per thread, then all key reads, then the (rare) atomics
    {
        bool bad = false;
        const int64_t P = 2 * m;
        const int64_t lo = P * t / T, hi = P * (t + 1) / T;
        const int32_t *srcg = a.src + E0, *dstg = a.dst + E0;
        // Idx: the type of the position indices.  32-bit indices save the
        // second instruction of every 64-bit add and compare; they are used
        // when no index of the sweep, counter steps included, can pass 2^32.
        auto sweep = [&](auto idx_tag) {
            using Idx = decltype(idx_tag);
            const Idx hi_ = (Idx)hi, m_ = (Idx)m;
            for (Idx b0 = (Idx)lo + (Idx)tid; b0 < hi_; b0 += (Idx)(kU * kBB)) {
                int32_t v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const Idx i = b0 + (Idx)(u * kBB);
                    v[u] = -1;
                    if (i < hi_) v[u] = i < m_ ? __ldcs(srcg + i) : __ldcs(dstg + (i - m_));
                }
                uint32_t own[kU], li[kU], cur[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const Idx i = b0 + (Idx)(u * kBB);
                    // predicates rather than branches; one CTA owns every vertex
                    const bool ok = i < hi_ && (uint32_t)v[u] < nn;
                    bad |= i < hi_ && !ok;
                    if constexpr (T == 1) {
                        own[u] = ok ? 0u : (uint32_t)kTeam;          // kTeam: "skip"
                        li[u] = (uint32_t)v[u];
                    } else {
                        own[u] = ok ? (uint32_t)v[u] / chunk : (uint32_t)kTeam;
                        li[u] = (uint32_t)v[u] - own[u] * chunk;
                    }
                    cur[u] = ok ? key_ptr<T>(s_keys, ts, own[u])[li[u]] : 0u;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t i = (uint32_t)(b0 + (Idx)(u * kBB));
                    if (own[u] < kTeam && cur[u] > i)
                        atomicMin(key_ptr<T>(s_keys, ts, own[u]) + li[u], i);
                }
            }
        };
        if (hi <= (int64_t)0xFFFFFFFFu - (int64_t)kU * kBB) sweep(uint32_t{});
        else sweep(int64_t{});
        if (bad) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
    }
    team_sync<T>(cl);

    // 3. mark first-occurrence positions; count vertices on no edge
    uint32_t iso = 0;
    for (int64_t i = tid; i < myn; i += kBB) {
        const uint32_t k = s_keys[i];
        if (k == kSent) { ++iso; continue; }
        const uint32_t w = k >> 5;                  // keys are 32-bit positions
        const uint32_t r = owner_of_word<T>(w, Wc);
        atomicOr(a.scratch + (cta0 + r) * a.region_words + (w - r * (uint32_t)Wc),
                 1u << (k & 31u));
    }
    {
        uint32_t tot;
        BlockScan<kBB>::exclusive(iso, &tot, ts.scan);
        if (tid == 0) ts.xiso = tot;
    }
    team_sync<T>(cl);

    // 4. popcount prefix of this member's bitmap slice, one value per 8 words
    {
        uint32_t carry = 0;
        for (int64_t cb = 0; cb < Wc; cb += (int64_t)kBB * 8) {
            const int64_t w0 = cb + (int64_t)tid * 8;
            uint32_t c = 0;
            if (w0 < Wc) {
                const uint4 x0 = __ldcg(reinterpret_cast<const uint4 *>(my_bm + w0));
                const uint4 x1 = __ldcg(reinterpret_cast<const uint4 *>(my_bm + w0) + 1);
                c = __popc(x0.x) + __popc(x0.y) + __popc(x0.z) + __popc(x0.w) + __popc(x1.x) +
                    __popc(x1.y) + __popc(x1.z) + __popc(x1.w);
            }
            uint32_t tot;
            const uint32_t ex = BlockScan<kBB>::exclusive(c, &tot, ts.scan);
            if (w0 < Wc) my_grp[w0 >> 3] = carry + ex;
            carry += tot;
        }
        if (tid == 0) ts.xtot = carry;
    }
    team_sync<T>(cl);
    if (tid == 0) {
        uint32_t K = 0, isob = 0;
        for (int r = 0; r < T; ++r) {
            uint32_t tr, ir;
            if constexpr (T == 1) { tr = ts.xtot; ir = ts.xiso; }
            else {
                tr = *cl->map_shared_rank(&ts.xtot, r);
                ir = *cl->map_shared_rank(&ts.xiso, r);
            }
            ts.base[r] = K;
            K += tr;
            if (r < t) isob += ir;
        }
        ts.on_edges = K;
        ts.iso_before = isob;
    }
    __syncthreads();

    // 5. labels, written over the keys; perm
    {
        const uint32_t K = ts.on_edges, isob = ts.iso_before;
        uint32_t carry = 0;
        for (int64_t ib = 0; ib < myn; ib += kBB) {
            const int64_t i = ib + tid;
            const uint32_t k = i < myn ? s_keys[i] : 0u;
            const uint32_t isf = (i < myn && k == kSent) ? 1u : 0u;
            uint32_t tot;
            const uint32_t ex = BlockScan<kBB>::exclusive(isf, &tot, ts.scan);
            if (i < myn) {
                uint32_t lab;
                if (isf) {
                    lab = K + isob + carry + ex;
                } else {
                    const uint32_t w = k >> 5;
                    const uint32_t r = owner_of_word<T>(w, Wc);
                    const uint32_t wl = w - r * (uint32_t)Wc;
                    const uint32_t *bm = a.scratch + (cta0 + r) * a.region_words;
                    const uint32_t *gp = bm + a.wmax;
                    const uint4 *gw = reinterpret_cast<const uint4 *>(bm + ((wl >> 3) << 3));
                    const uint4 q0 = __ldcg(gw), q1 = __ldcg(gw + 1);
                    const uint32_t ws[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                    const uint32_t wi = (uint32_t)(wl & 7);
                    lab = ts.base[r] + __ldcg(gp + (wl >> 3));
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if ((uint32_t)j < wi) lab += __popc(ws[j]);
                        else if ((uint32_t)j == wi) lab += __popc(ws[j] & ((1u << (k & 31u)) - 1u));
                    }
                }
                s_keys[i] = lab;
                if (lab < nn) a.perm[V0 + lab] = (int32_t)(v_lo + i);
                else raise_status(a.status, BOBA_ERR_TIMEOUT);
            }
            carry += tot;
        }
    }
    team_sync<T>(cl);

    // 6. relabel this member's share of the edges: kU/2 edges (kU loads) in
    // flight per thread, all label reads, then the stores
    {
        constexpr int U2 = kU / 2;
        // 32-bit edge indices: hi <= m < 2^31, so no counter step passes 2^32
        const uint32_t lo = (uint32_t)(m * t / T), hi = (uint32_t)(m * (t + 1) / T);
        const int32_t *srcg = a.src + E0, *dstg = a.dst + E0;
        int32_t *sog = a.so + E0, *dog = a.dout + E0;
        for (uint32_t b0 = lo + (uint32_t)tid; b0 < hi; b0 += (uint32_t)(U2 * kBB)) {
            int32_t v[kU];
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const uint32_t e = b0 + (uint32_t)(u * kBB);
                v[2 * u] = v[2 * u + 1] = -1;
                if (e < hi) {
                    v[2 * u] = __ldcs(srcg + e);
                    v[2 * u + 1] = __ldcs(dstg + e);
                }
            }
            int32_t lab[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const bool ok = (uint32_t)v[u] < nn;
                uint32_t o = 0, l = (uint32_t)v[u];
                if constexpr (T > 1) {
                    o = ok ? (uint32_t)v[u] / chunk : 0u;
                    l = (uint32_t)v[u] - o * chunk;
                }
                lab[u] = ok ? (int32_t)key_ptr<T>(s_keys, ts, o)[l] : -1;
            }
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const uint32_t e = b0 + (uint32_t)(u * kBB);
                if (e >= hi) continue;
                if (lab[2 * u] < 0 || lab[2 * u + 1] < 0)
                    raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                __stcs(sog + e, lab[2 * u]);
                __stcs(dog + e, lab[2 * u + 1]);
            }
        }
    }
    team_sync<T>(cl);    // nobody leaves while a member may still read its labels
}

__global__ void __cluster_dims__(kTeam, 1, 1) __launch_bounds__(kBB, 1) k_batch(BatchArgs a)
{
    extern __shared__ uint32_t s_keys[];
    __shared__ TeamSmem ts;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int64_t cluster_cta0 = (int64_t)blockIdx.x - rank;
    while (true) {
        if (rank == 0 && threadIdx.x == 0) ts.item = atomicAdd(&a.hdr[kHdrTicket], 1u);
        cl.sync();
        const uint32_t item = *cl.map_shared_rank(&ts.item, 0);
        cl.sync();
        const uint32_t n_items = a.hdr[kHdrItems];
        if (item >= n_items) break;
        const uint32_t n_large = a.hdr[kHdrLarge];
        if (item < n_large) {
            process_graph<kTeam>(a, a.order[item], rank, cluster_cta0, &cl, s_keys, ts);
        } else {
            const uint32_t idx = n_large + (item - n_large) * kTeam + (uint32_t)rank;
            if (idx < a.hdr[kHdrValid])
                process_graph<1>(a, a.order[idx], 0, (int64_t)blockIdx.x, nullptr, s_keys, ts);
        }
    }
}

// Split mode, small graphs: one CTA per graph, persistent, no clusters.
__global__ void __launch_bounds__(kBB, 1) k_batch_small(BatchArgs a)
{
    extern __shared__ uint32_t s_keys[];
    __shared__ TeamSmem ts;
    const uint32_t n_large = a.hdr[kHdrLarge], n_valid = a.hdr[kHdrValid];
    while (true) {
        if (threadIdx.x == 0) ts.item = atomicAdd(&a.hdr[kHdrTicket], 1u);
        __syncthreads();
        const uint32_t idx = n_large + ts.item;
        __syncthreads();
        if (idx >= n_valid) break;
        process_graph<1>(a, a.order[idx], 0, (int64_t)blockIdx.x, nullptr, s_keys, ts);
    }
}

// ---------------------------------------------------------------------------
// Split mode, large graphs: all of them together, phase by phase.
// ---------------------------------------------------------------------------

// Largest j in [0, L) with tab[j] <= x (tab[0] = 0, tab[L] = total, x < total).
__device__ __forceinline__ uint32_t find_graph(const uint32_t *__restrict__ tab, uint32_t L, uint32_t x)
{
    uint32_t lo = 0, hi = L;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(tab + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

struct LargeItem {
    uint32_t j;              // index among the large graphs
    int64_t E0, m, V0, n;
    uint32_t local;          // chunk / tile index within the graph
};

// The graph that owns item x.  A block's items only move forward, so thread 0
// first tries the graph of its previous item (`hint`) and the next few before
// falling back to a binary search over all large graphs.
__device__ __forceinline__ void block_find(const BatchArgs &a, const uint32_t *tab, uint32_t x,
                                           LargeItem &it, LargeItem &s_it, uint32_t &hint)
{
    if (threadIdx.x == 0) {
        const uint32_t L = a.hdr[kHdrLarge];
        uint32_t j = hint;
        bool found = false;
        for (int k = 0; k < 4 && j < L; ++k, ++j) {
            const uint32_t lo = __ldg(tab + j);
            if (lo > x) break;
            if (x < __ldg(tab + j + 1)) { found = true; break; }
        }
        if (!found) j = find_graph(tab, L, x);
        hint = j;
        s_it.j = j;
        const uint32_t g = a.order[s_it.j];
        s_it.E0 = a.eoff[g];
        s_it.m = a.eoff[g + 1] - s_it.E0;
        s_it.V0 = a.voff[g];
        s_it.n = a.voff[g + 1] - s_it.V0;
        s_it.local = x - tab[s_it.j];
    }
    __syncthreads();
    it = s_it;
    __syncthreads();
}

__global__ void __launch_bounds__(kLB) k_bl_init(BatchArgs a)
{
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t vt = a.lg_vt[L], wt = a.lg_wt[L];
    // keys of every large graph = SENT (padding too), clear bitmaps and scan state
    const int64_t stride = (int64_t)gridDim.x * kLB;
    const uint4 sent = make_uint4(kSent, kSent, kSent, kSent), z = make_uint4(0, 0, 0, 0);
    for (int64_t i = (int64_t)blockIdx.x * kLB + threadIdx.x; i < (int64_t)vt * kVtxTile / 4; i += stride)
        reinterpret_cast<uint4 *>(a.kl)[i] = sent;
    for (int64_t i = (int64_t)blockIdx.x * kLB + threadIdx.x; i < (int64_t)wt * kWordTile / 4; i += stride)
        reinterpret_cast<uint4 *>(a.lbm)[i] = z;
    for (int64_t i = (int64_t)blockIdx.x * kLB + threadIdx.x; i < wt; i += stride) a.lts_scan[i] = 0;
    for (int64_t i = (int64_t)blockIdx.x * kLB + threadIdx.x; i < vt; i += stride) a.lts_emit[i] = 0;
}

__global__ void __launch_bounds__(kLB) k_bl_first(BatchArgs a)
{
    __shared__ LargeItem s_it;
    uint32_t hint = 0;                     // thread 0: graph of the previous item
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_pc[L];
    constexpr int U = 16;                  // positions per thread per round
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        LargeItem it;
        block_find(a, a.lg_pc, c, it, s_it, hint);
        if (cdiv(it.n, kKcap) <= a.first_smax) continue;      // done by the sliced kernel
        const uint32_t nn = (uint32_t)it.n;
        uint32_t *key = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
        const int64_t c0 = (int64_t)it.local * kPosChunk;
        const int64_t p1 = min(c0 + (int64_t)kPosChunk, 2 * it.m);
        for (int64_t p0 = c0; p0 < p1; p0 += (int64_t)U * kLB) {
            int32_t v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = p0 + u * kLB + threadIdx.x;
                v[u] = -1;
                if (i < p1)
                    v[u] = i < it.m ? __ldcs(a.src + it.E0 + i) : __ldcs(a.dst + it.E0 + (i - it.m));
            }
            uint32_t cur[U];
#pragma unroll
            for (int u = 0; u < U; ++u) cur[u] = (uint32_t)v[u] < nn ? key[v[u]] : 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = p0 + u * kLB + threadIdx.x;
                if (i >= p1) continue;
                if ((uint32_t)v[u] >= nn) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                else if (cur[u] > (uint32_t)i) atomicMin(&key[v[u]], (uint32_t)i);
            }
        }
    }
}

// Locate chunk c of the table `tab` for one warp: lane 0 searches (from the
// warp's previous graph, `hint`) and publishes the item in `slot`.
__device__ __forceinline__ LargeItem warp_find(const BatchArgs &a, const uint32_t *tab, uint32_t L,
                                               uint32_t c, LargeItem &slot, uint32_t &hint)
{
    if ((threadIdx.x & 31) == 0) {
        uint32_t j = hint;
        bool found = false;
        for (int k = 0; k < 4 && j < L; ++k, ++j) {
            if (__ldg(tab + j) > c) break;
            if (c < __ldg(tab + j + 1)) { found = true; break; }
        }
        if (!found) j = find_graph(tab, L, c);
        hint = j;
        const uint32_t g = a.order[j];
        slot.j = j;
        slot.E0 = a.eoff[g];
        slot.m = a.eoff[g + 1] - slot.E0;
        slot.V0 = a.voff[g];
        slot.n = a.voff[g + 1] - slot.V0;
        slot.local = c - tab[j];
    }
    __syncwarp();
    const LargeItem it = slot;
    __syncwarp();                          // the slot is rewritten for the next chunk
    return it;
}

// Runs of consecutive chunks for one CTA per SM: the block claims run r from
// `ticket`; returns false once all `runs` are taken.
__device__ __forceinline__ bool claim_run(uint32_t *ticket, uint32_t runs, uint32_t &s_run,
                                          uint32_t &r)
{
    if (threadIdx.x == 0) s_run = atomicAdd(ticket, 1u);
    __syncthreads();
    r = s_run;
    __syncthreads();                       // s_run is rewritten for the next run
    return r < runs;
}

constexpr int kRunBlock = 1024;
constexpr int kRunWarps = kRunBlock / 32;
constexpr uint32_t kRunPosChunks = 128;          // 2 M positions per run

// The global first-occurrence pass in runs (see k_bl_relabel_runs): an SM
// works on one graph's key array at a time, so the filtering reads of keys
// already lowered can hit its L1.  A filtering read that L1 serves may be
// older than the key in L2; keys only decrease, so it is never below the
// current key and at worst costs an atomicMin that changes nothing.
__global__ void __launch_bounds__(kRunBlock, 1) k_bl_first_runs(BatchArgs a)
{
    __shared__ uint32_t s_run;
    __shared__ LargeItem s_it[kRunWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t hint = 0;
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_pc[L];
    const uint32_t runs = (total + kRunPosChunks - 1) / kRunPosChunks;
    constexpr int U = 16;                       // positions per lane per round
    constexpr int kRound = 32 * U;
    static_assert(kPosChunk % kRound == 0, "a chunk is whole rounds of a warp");
    uint32_t r;
    while (claim_run(&a.hdr[kHdrFirstRunTicket], runs, s_run, r)) {
        const uint32_t cend = min(total, (r + 1) * kRunPosChunks);
        for (uint32_t c = r * kRunPosChunks + w; c < cend; c += kRunWarps) {
            const LargeItem it = warp_find(a, a.lg_pc, L, c, s_it[w], hint);
            if (cdiv(it.n, kKcap) <= a.first_smax) continue;      // done by the sliced kernel
            const uint32_t nn = (uint32_t)it.n;
            uint32_t *key = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
            const int64_t c0 = (int64_t)it.local * kPosChunk;
            const int64_t p1 = min(c0 + (int64_t)kPosChunk, 2 * it.m);
            for (int64_t base = c0; base < p1; base += kRound) {
                int32_t v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t i = base + u * 32 + lane;
                    v[u] = -1;
                    if (i < p1)
                        v[u] = i < it.m ? __ldcs(a.src + it.E0 + i)
                                        : __ldcs(a.dst + it.E0 + (i - it.m));
                }
                uint32_t cur[U];
#pragma unroll
                for (int u = 0; u < U; ++u) cur[u] = (uint32_t)v[u] < nn ? key[v[u]] : 0u;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t i = base + u * 32 + lane;
                    if (i >= p1) continue;
                    if ((uint32_t)v[u] >= nn) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                    else if (cur[u] > (uint32_t)i) atomicMin(&key[v[u]], (uint32_t)i);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kLB) k_bl_mark(BatchArgs a)
{
    __shared__ LargeItem s_it;
    uint32_t hint = 0;                     // thread 0: graph of the previous item
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_vt[L];
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        LargeItem it;
        block_find(a, a.lg_vt, c, it, s_it, hint);
        const uint32_t *key = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
        uint32_t *bm = a.lbm + (size_t)a.lg_wt[it.j] * kWordTile;
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            const int64_t v0 = (int64_t)it.local * kVtxTile + r * kVtxRow + 4 * threadIdx.x;
            const uint4 k4 = *reinterpret_cast<const uint4 *>(key + v0);
            const uint32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (v0 + q < it.n && kk[q] != kSent) atomicOr(&bm[kk[q] >> 5], 1u << (kk[q] & 31u));
        }
    }
}

__global__ void __launch_bounds__(kLB) k_bl_scan(BatchArgs a)
{
    __shared__ LargeItem s_it;
    uint32_t hint = 0;                     // thread 0: graph of the previous item
    __shared__ typename BlockScan<kLB>::Smem sm;
    __shared__ uint32_t s_rowtot[kBlRows];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_pre;
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_wt[L];
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&a.hdr[kHdrScanTicket], 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        __syncthreads();
        if (t >= total) break;
        LargeItem it;
        block_find(a, a.lg_wt, t, it, s_it, hint);
        // row r of the tile: words t*kWordTile + r*kWordRow .., this thread's sector at 8*tid
        uint32_t within[kBlRows];
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            const size_t w0 = (size_t)t * kWordTile + r * kWordRow + 8 * threadIdx.x;
            const uint4 x0 = __ldcg(reinterpret_cast<const uint4 *>(a.lbm + w0));
            const uint4 x1 = __ldcg(reinterpret_cast<const uint4 *>(a.lbm + w0) + 1);
            const uint32_t c = __popc(x0.x) + __popc(x0.y) + __popc(x0.z) + __popc(x0.w) +
                               __popc(x1.x) + __popc(x1.y) + __popc(x1.z) + __popc(x1.w);
            uint32_t rt;
            within[r] = BlockScan<kLB>::exclusive(c, &rt, sm);
            if (threadIdx.x == 0) s_rowtot[r] = rt;
            __syncthreads();               // the scan's shared words are reused
        }
        uint32_t before[kBlRows], tot = 0;
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            before[r] = tot + within[r];
            tot += s_rowtot[r];
        }
        if (threadIdx.x < 32) {
            const uint64_t p = lookback_exclusive(a.lts_scan, t, tot, a.status, it.local == 0);
            if (threadIdx.x == 0) s_pre = p;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kBlRows; ++r)
            a.lgrp[((size_t)t * kWordTile + r * kWordRow + 8 * threadIdx.x) >> 3] =
                (uint32_t)s_pre + before[r];
        if (threadIdx.x == 0 && t + 1 == a.lg_wt[it.j + 1]) a.lg_tot[it.j] = (uint32_t)s_pre + tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kLB) k_bl_emit(BatchArgs a)
{
    __shared__ LargeItem s_it;
    uint32_t hint = 0;                     // thread 0: graph of the previous item
    __shared__ typename BlockScan<kLB>::Smem sm;
    __shared__ uint32_t s_rowtot[kBlRows];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_pre;
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_vt[L];
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&a.hdr[kHdrEmitTicket], 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        __syncthreads();
        if (t >= total) break;
        LargeItem it;
        block_find(a, a.lg_vt, t, it, s_it, hint);
        uint32_t *key = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
        const size_t wbase = (size_t)a.lg_wt[it.j] * kWordTile;
        // row r of the tile: vertices local*kVtxTile + r*kVtxRow .., this
        // thread's four at 4*tid; vertex order is row-major
        uint32_t kk[kBlRows][4], within[kBlRows];
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            const int64_t v0 = (int64_t)it.local * kVtxTile + r * kVtxRow + 4 * threadIdx.x;
            const uint4 k4 = *reinterpret_cast<const uint4 *>(key + v0);
            kk[r][0] = k4.x;
            kk[r][1] = k4.y;
            kk[r][2] = k4.z;
            kk[r][3] = k4.w;
            uint32_t c = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) c += (v0 + q < it.n && kk[r][q] == kSent) ? 1u : 0u;
            uint32_t rt;
            within[r] = BlockScan<kLB>::exclusive(c, &rt, sm);
            if (threadIdx.x == 0) s_rowtot[r] = rt;
            __syncthreads();               // the scan's shared words are reused
        }
        uint32_t before[kBlRows], tot = 0;
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            before[r] = tot + within[r];
            tot += s_rowtot[r];
        }
        if (threadIdx.x < 32) {
            const uint64_t p = lookback_exclusive(a.lts_emit, t, tot, a.status, it.local == 0);
            if (threadIdx.x == 0) s_pre = p;
        }
        __syncthreads();
        const uint32_t K = __ldcg(a.lg_tot + it.j);
#pragma unroll
        for (int r = 0; r < kBlRows; ++r) {
            const int64_t v0 = (int64_t)it.local * kVtxTile + r * kVtxRow + 4 * threadIdx.x;
            uint32_t next_iso = K + (uint32_t)s_pre + before[r];
            uint32_t lab[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                lab[q] = kSent;
                if (v0 + q >= it.n) continue;
                if (kk[r][q] == kSent) {
                    lab[q] = next_iso++;
                } else {
                    const uint32_t k = kk[r][q];
                    const size_t gidx = (wbase >> 3) + (k >> 8);
                    const uint4 *gw = reinterpret_cast<const uint4 *>(a.lbm + (gidx << 3));
                    const uint4 q0 = __ldcg(gw), q1 = __ldcg(gw + 1);
                    const uint32_t ws[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                    const uint32_t wi = (k >> 5) & 7u;
                    uint32_t rk = __ldcg(a.lgrp + gidx);      // prefixes restart at each graph
#pragma unroll
                    for (int i2 = 0; i2 < 8; ++i2) {
                        if ((uint32_t)i2 < wi) rk += __popc(ws[i2]);
                        else if ((uint32_t)i2 == wi) rk += __popc(ws[i2] & ((1u << (k & 31u)) - 1u));
                    }
                    lab[q] = rk;
                }
                if (lab[q] < (uint32_t)it.n) a.perm[it.V0 + lab[q]] = (int32_t)(v0 + q);
                else raise_status(a.status, BOBA_ERR_TIMEOUT);
            }
            *reinterpret_cast<uint4 *>(key + v0) = make_uint4(lab[0], lab[1], lab[2], lab[3]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kLB) k_bl_relabel(BatchArgs a)
{
    __shared__ LargeItem s_it;
    uint32_t hint = 0;                     // thread 0: graph of the previous item
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_ec[L];
    constexpr int U = 8;                   // edges per thread per round
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        LargeItem it;
        block_find(a, a.lg_ec, c, it, s_it, hint);
        if (cdiv(it.n, kKcap) <= a.relabel_smax) continue;    // done by the sliced kernel
        const uint32_t nn = (uint32_t)it.n;
        const uint32_t *lab = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
        const int64_t c0 = (int64_t)it.local * kEdgeChunk;
        const int64_t c1 = min(c0 + (int64_t)kEdgeChunk, it.m);
        for (int64_t e0 = c0; e0 < c1; e0 += (int64_t)U * kLB) {
            int32_t s[U], d[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e0 + u * kLB + threadIdx.x;
                s[u] = d[u] = -1;
                if (e < c1) {
                    s[u] = __ldcs(a.src + it.E0 + e);
                    d[u] = __ldcs(a.dst + it.E0 + e);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                s[u] = (uint32_t)s[u] < nn ? (int32_t)__ldg(lab + s[u]) : -1;
                d[u] = (uint32_t)d[u] < nn ? (int32_t)__ldg(lab + d[u]) : -1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e0 + u * kLB + threadIdx.x;
                if (e >= c1) continue;
                if (s[u] < 0 || d[u] < 0) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                __stcs(a.so + it.E0 + e, s[u]);
                __stcs(a.dout + it.E0 + e, d[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Sliced large path: for large graphs of at most kMaxSlices * kKcap vertices,
// the first-occurrence and relabel phases run with the keys (labels) in
// shared memory.  A graph's vertex range is cut into slices of kKcap; task
// (graph, slice) is one persistent CTA's: it streams all of the graph's
// endpoints and handles only those in its slice.  A graph's slices are
// consecutive tasks, so they run side by side and read the same lines: the
// streams are loaded with normal L2 priority so that only the first slice
// reads them from DRAM.  Every key / label access is a shared-memory access
// instead of an L1/L2 gather.  The bitmap, scan and emit phases between them are the ones above.
// ---------------------------------------------------------------------------

constexpr int kSliceU = 8;                 // int4 stream loads in flight per thread

// Calls f(v, p) for every element v = X[e], e in [0, m), with p = pos0 + e:
// a head of up to three elements to the next 16-byte boundary, the body in
// int4 loads, and a tail of up to three.  Indices and positions fit in 32
// bits (2m < 2^32), which keeps the per-element work short.
template <class F>
__device__ __forceinline__ void stream_block(const int32_t *__restrict__ X, int64_t m, int64_t pos0,
                                             F f)
{
    const uint32_t mm = (uint32_t)m, p0 = (uint32_t)pos0;
    uint32_t head = ((16u - ((uint32_t)(uintptr_t)X & 15u)) & 15u) >> 2;
    if (head > mm) head = mm;
    if (threadIdx.x < head) f(__ldcg(X + threadIdx.x), p0 + threadIdx.x);
    const int4 *X4 = reinterpret_cast<const int4 *>(X + head);
    const uint32_t q = (mm - head) >> 2;
    const uint32_t pb = p0 + head;
    constexpr uint32_t step = (uint32_t)kBB * kSliceU;
    for (uint32_t b0 = threadIdx.x; b0 < q; b0 += step) {
        int4 w[kSliceU];
#pragma unroll
        for (int u = 0; u < kSliceU; ++u) {
            const uint32_t k = b0 + (uint32_t)u * kBB;
            w[u] = k < q ? __ldcg(X4 + k) : make_int4(-1, -1, -1, -1);   // kept in L2 for the sibling slices
        }
#pragma unroll
        for (int u = 0; u < kSliceU; ++u) {
            const uint32_t k = b0 + (uint32_t)u * kBB;
            if (k < q) {
                const uint32_t p = pb + 4u * k;
                f(w[u].x, p);
                f(w[u].y, p + 1u);
                f(w[u].z, p + 2u);
                f(w[u].w, p + 3u);
            }
        }
    }
    const uint32_t t0 = head + 4u * q;
    if (t0 + threadIdx.x < mm) f(__ldcg(X + t0 + threadIdx.x), p0 + t0 + threadIdx.x);
}

// The sliced first-occurrence visit of X[0, m) at positions pos0 + e, for the
// slice [base, base + cnt) whose keys are in s_keys.  Per group of
// kFirstSliceG int4 loads, every element's filtering read of its key is issued
// before any atomicMin: an atomic may alias a later read, so interleaving them
// would serialise each element on the shared-memory latency.  A key read early
// may be stale; keys only decrease, so it is never below the current key and
// at worst costs an atomicMin that changes nothing.  With CHECK, vmax takes
// the largest ID seen (as unsigned, so a negative ID counts as huge).
constexpr int kFirstSliceU = 6;
constexpr int kFirstSliceG = 2;                 // int4 loads per read-then-update group
static_assert(kFirstSliceU % kFirstSliceG == 0, "whole groups");

__device__ __forceinline__ int32_t lane_of(const int4 &q, int j)
{
    return j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
}

template <bool CHECK>
__device__ __forceinline__ void first_slice_stream(const int32_t *__restrict__ X, int64_t m,
                                                   int64_t pos0, uint32_t base, uint32_t cnt,
                                                   uint32_t *s_keys, uint32_t &vmax)
{
    const uint32_t mm = (uint32_t)m, p0 = (uint32_t)pos0;
    auto one = [&](int32_t v, uint32_t p) {
        const uint32_t u = (uint32_t)v - base;
        const bool own = u < cnt;
        const uint32_t cur = own ? s_keys[u] : 0u;
        if (own && cur > p) atomicMin(&s_keys[u], p);
        if constexpr (CHECK) vmax = max(vmax, (uint32_t)v);
    };
    uint32_t head = ((16u - ((uint32_t)(uintptr_t)X & 15u)) & 15u) >> 2;
    if (head > mm) head = mm;
    if (threadIdx.x < head) one(__ldcg(X + threadIdx.x), p0 + threadIdx.x);
    const int4 *X4 = reinterpret_cast<const int4 *>(X + head);
    const uint32_t q = (mm - head) >> 2;
    const uint32_t pb = p0 + head;
    constexpr uint32_t step = (uint32_t)kBB * kFirstSliceU;
    for (uint32_t b0 = threadIdx.x; b0 < q; b0 += step) {
        int4 w[kFirstSliceU];
#pragma unroll
        for (int u = 0; u < kFirstSliceU; ++u) {
            const uint32_t k = b0 + (uint32_t)u * kBB;
            // -1 beyond the end: outside every slice, and not counted in vmax
            w[u] = k < q ? __ldcg(X4 + k) : make_int4(-1, -1, -1, -1);   // kept in L2 for the sibling slices
        }
        // the filtering reads, then the atomics, for kFirstSliceG of the
        // loads at a time (registers: the reads of all of them would not fit)
#pragma unroll
        for (int h = 0; h < kFirstSliceU; h += kFirstSliceG) {
            uint32_t cur[4 * kFirstSliceG];
#pragma unroll
            for (int u = h; u < h + kFirstSliceG; ++u) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t x = (uint32_t)lane_of(w[u], j) - base;
                    cur[4 * (u - h) + j] = x < cnt ? s_keys[x] : 0u;
                    if constexpr (CHECK)
                        if (b0 + (uint32_t)u * kBB < q) vmax = max(vmax, (uint32_t)lane_of(w[u], j));
                }
            }
            // an endpoint outside the slice read 0, which no position is below
#pragma unroll
            for (int u = h; u < h + kFirstSliceG; ++u) {
                const uint32_t p = pb + 4u * (b0 + (uint32_t)u * kBB);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (cur[4 * (u - h) + j] > p + (uint32_t)j)
                        atomicMin(&s_keys[(uint32_t)lane_of(w[u], j) - base], p + (uint32_t)j);
            }
        }
    }
    const uint32_t t0 = head + 4u * q;
    if (t0 + threadIdx.x < mm) one(__ldcg(X + t0 + threadIdx.x), p0 + t0 + threadIdx.x);
}

__global__ void __launch_bounds__(kBB, 1) k_bl_first_sliced(BatchArgs a)
{
    extern __shared__ uint32_t s_keys[];   // kKcap
    __shared__ LargeItem s_it;
    __shared__ uint32_t s_task;
    uint32_t hint = 0;                     // thread 0: graph of the previous task
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_st[L];
    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(&a.hdr[kHdrSliceFirst], 1u);
        __syncthreads();
        const uint32_t t = s_task;
        if (t >= total) break;
        LargeItem it;
        block_find(a, a.lg_st, t, it, s_it, hint);
        if (cdiv(it.n, kKcap) > a.first_smax) continue;       // done by the global kernel
        const uint32_t base = it.local * (uint32_t)kKcap;
        const uint32_t cnt = (uint32_t)min((int64_t)kKcap, it.n - base);
        for (uint32_t i = threadIdx.x; i < cnt; i += kBB) s_keys[i] = kSent;
        __syncthreads();
        // few branches per element: most endpoints belong to other slices,
        // and divergent branches cost more here than the predicated load.
        // An ID outside [0, n) is in no slice, so it is never written; the
        // task of slice 0 alone looks for one, as the largest ID it sees.
        uint32_t vmax = 0;
        if (it.local == 0) {
            first_slice_stream<true>(a.src + it.E0, it.m, 0, base, cnt, s_keys, vmax);
            first_slice_stream<true>(a.dst + it.E0, it.m, it.m, base, cnt, s_keys, vmax);
            if (vmax >= (uint32_t)it.n) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
        } else {
            first_slice_stream<false>(a.src + it.E0, it.m, 0, base, cnt, s_keys, vmax);
            first_slice_stream<false>(a.dst + it.E0, it.m, it.m, base, cnt, s_keys, vmax);
        }
        __syncthreads();
        uint32_t *key = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile + base;
        for (uint32_t i = threadIdx.x; i < cnt; i += kBB) key[i] = s_keys[i];
        __syncthreads();                   // s_keys and s_task are reused
    }
}

// The global relabel with the work claimed in runs of kRunChunks consecutive
// chunks by one 1024-thread CTA per SM.  A run lies mostly inside one graph, so
// while an SM works through it its L1 holds much of that graph's label array
// (up to 1 MB for the graphs of this path): a label lookup that hits L1 sends
// no request to L2, and the lookups are bound by that request rate.  In the
// grid-stride kernel above, an SM's blocks work on unrelated graphs at once.
// A ticket hands out the runs, so the SMs stay balanced.  Inside a run each
// warp takes every 32nd chunk on its own, with no block-wide barrier.
constexpr uint32_t kRunChunks = 256;            // 2 M edges per run

__global__ void __launch_bounds__(kRunBlock, 1) k_bl_relabel_runs(BatchArgs a)
{
    __shared__ uint32_t s_run;
    __shared__ LargeItem s_it[kRunWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t hint = 0;
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_ec[L];
    const uint32_t runs = (total + kRunChunks - 1) / kRunChunks;
    constexpr int U = 8;                        // edges per lane per round
    constexpr int kRound = 32 * U;
    static_assert(kEdgeChunk % kRound == 0, "a chunk is whole rounds of a warp");
    uint32_t r;
    while (claim_run(&a.hdr[kHdrRunTicket], runs, s_run, r)) {
        const uint32_t cend = min(total, (r + 1) * kRunChunks);
        for (uint32_t c = r * kRunChunks + w; c < cend; c += kRunWarps) {
            const LargeItem it = warp_find(a, a.lg_ec, L, c, s_it[w], hint);
            if (cdiv(it.n, kKcap) <= a.relabel_smax) continue;    // done by the sliced kernel
            const uint32_t nn = (uint32_t)it.n;
            const uint32_t *lab = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile;
            const int64_t c0 = (int64_t)it.local * kEdgeChunk;
            const int64_t c1 = min(c0 + (int64_t)kEdgeChunk, it.m);
            for (int64_t base = c0; base < c1; base += kRound) {
                int32_t sv[U], dv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t e = base + u * 32 + lane;
                    sv[u] = dv[u] = -1;
                    if (e < c1) {
                        sv[u] = __ldcs(a.src + it.E0 + e);
                        dv[u] = __ldcs(a.dst + it.E0 + e);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    sv[u] = (uint32_t)sv[u] < nn ? (int32_t)__ldg(lab + sv[u]) : -1;
                    dv[u] = (uint32_t)dv[u] < nn ? (int32_t)__ldg(lab + dv[u]) : -1;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t e = base + u * 32 + lane;
                    if (e >= c1) continue;
                    if (sv[u] < 0 || dv[u] < 0) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                    __stcs(a.so + it.E0 + e, sv[u]);
                    __stcs(a.dout + it.E0 + e, dv[u]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kBB, 1) k_bl_relabel_sliced(BatchArgs a)
{
    extern __shared__ uint32_t s_lab[];    // kKcap
    __shared__ LargeItem s_it;
    __shared__ uint32_t s_task;
    uint32_t hint = 0;
    const uint32_t L = a.hdr[kHdrLarge];
    const uint32_t total = a.lg_st[L];
    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(&a.hdr[kHdrSliceRelabel], 1u);
        __syncthreads();
        const uint32_t t = s_task;
        if (t >= total) break;
        LargeItem it;
        block_find(a, a.lg_st, t, it, s_it, hint);
        if (cdiv(it.n, kKcap) > a.relabel_smax) continue;     // done by the global kernel
        const uint32_t base = it.local * (uint32_t)kKcap;
        const uint32_t cnt = (uint32_t)min((int64_t)kKcap, it.n - base);
        const uint32_t *lab = a.kl + (size_t)a.lg_vt[it.j] * kVtxTile + base;
        for (uint32_t i = threadIdx.x; i < cnt; i += kBB) s_lab[i] = __ldcg(lab + i);
        __syncthreads();
        const uint32_t nn = (uint32_t)it.n;
        const bool first_slice = it.local == 0;
        bool bad = false;
        // each output element is written by the one task whose slice holds its
        // vertex (an ID outside [0, n) by the first slice, as -1); plain
        // stores, so that the slices' partial writes of one line merge in L2
        auto out = [&](int32_t *o) {
            return [&, o](int32_t v, uint32_t e) {
                const uint32_t u = (uint32_t)v - base;
                const bool own = u < cnt;
                const bool oob = (uint32_t)v >= nn;
                bad |= oob;
                if (own || (oob && first_slice)) o[e] = own ? (int32_t)s_lab[u] : -1;
            };
        };
        stream_block(a.src + it.E0, it.m, 0, out(a.so + it.E0));
        stream_block(a.dst + it.E0, it.m, 0, out(a.dout + it.E0));
        if (bad && first_slice) raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
        __syncthreads();                   // s_lab and s_task are reused
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct BatchDevice {
    bool ready = false;
    int grid_cluster = 0;    // CTAs of the persistent cluster launch
    int grid_small = 0;      // CTAs of the persistent non-cluster launch
    int sms = 0;
};
std::mutex g_bmu;
BatchDevice g_bdev[64];
int g_mode_override = -1;    // set by the autotuner API; -1 = default

const BatchDevice *batch_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchDevice &d = g_bdev[dev];
    if (!d.ready) {
        if (cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDynSmem) != cudaSuccess ||
            cudaFuncSetAttribute((const void *)k_batch_small,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDynSmem) != cudaSuccess ||
            cudaFuncSetAttribute((const void *)k_bl_first_sliced,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDynSmem) != cudaSuccess ||
            cudaFuncSetAttribute((const void *)k_bl_relabel_sliced,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDynSmem) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kTeam, 1, 1);
        cfg.blockDim = dim3(kBB, 1, 1);
        cfg.dynamicSmemBytes = kDynSmem;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)k_batch, &cfg) != cudaSuccess ||
            clusters < 1) {
            (void)cudaGetLastError();
            return nullptr;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_batch_small, kBB,
                                                          kDynSmem) != cudaSuccess || per_sm < 1) {
            (void)cudaGetLastError();
            return nullptr;
        }
        d.grid_cluster = clusters * kTeam;
        d.grid_small = d.sms * per_sm;
        d.ready = true;
    }
    return &d;
}

// Explicit setting, else the autotuned choice for this size, else the
// environment, else split.
int batch_mode(int64_t total_m)
{
    if (g_mode_override >= 0) return g_mode_override == 0 ? kBatchCluster : kBatchSplit;
    const int v = tuned_variant(kTuneBatched, total_m);      // 1 cluster, the others split
    if (v == 1) return kBatchCluster;
    const char *e = getenv("BOBA_BATCH_MODE");
    if (v == 0 && e && strcmp(e, "cluster") == 0) return kBatchCluster;
    return kBatchSplit;
}

// Split mode: up to how many slices a large graph takes the sliced
// first-occurrence (fs) and relabel (rs) kernel instead of the global one.
// Schedules (the numbers of boba_batched_set_mode; the tuner's variants are
// the same except that its 0 is schedule 6, its 1 schedule 0, its 6 schedule 1):
//   1: fs 8, rs 1 (a one-slice graph relabels without redundant streams or
//      partial writes; the global relabel strides over the chunks)
//   2: fs 8, rs 8     3: fs 8, rs 2     4: global phases only     5: fs 3, rs 0
//   6: as 1, with the global relabel claiming runs of chunks per SM (the
//      default: measured best on the 4096-graph batch, 28.1 ms against 31.1)
//   7: as 6, with the global first-occurrence pass in runs too
//   8: as 7 with fs 1
void batch_slices(int64_t total_m, int &fs, int &rs, bool &first_runs, bool &runs)
{
    int sched = g_mode_override;
    if (sched < 0) {
        const int v = tuned_variant(kTuneBatched, total_m);
        sched = v == 0 ? 6 : v == 1 ? 0 : v == 6 ? 1 : v;
    }
    fs = rs = 0;
    first_runs = runs = false;
    if (sched == 1) { fs = kMaxSlices; rs = 1; }
    else if (sched == 2) { fs = kMaxSlices; rs = kMaxSlices; }
    else if (sched == 3) { fs = kMaxSlices; rs = 2; }
    else if (sched == 5) { fs = 3; }
    else if (sched == 6) { fs = kMaxSlices; rs = 1; runs = true; }
    else if (sched == 7) { fs = kMaxSlices; rs = 1; first_runs = runs = true; }
    else if (sched == 8) { fs = 1; rs = 1; first_runs = runs = true; }
}

struct BatchLayout {
    int64_t wmax, region_words, regions, lvt_cap, lwt_cap;
    size_t hdr, order, scratch, tabs, kl, lbm, lgrp, lts_scan, lts_emit, total;
};

bool batch_layout(int64_t G, int64_t max_m, int64_t max_n, int64_t total_m, int64_t total_n,
                  const BatchDevice *d, int mode, BatchLayout &L)
{
    if (G < 0 || max_m < 0 || max_n < 0 || total_m < 0 || total_n < 0 || max_m > kMaxSize ||
        max_n > kMaxSize || d == nullptr)
        return false;
    // per-CTA bitmap regions: in split mode only graphs up to kSmallMaxM edges use them
    const int64_t region_m = mode == kBatchSplit ? (max_m < kSmallMaxM ? max_m : kSmallMaxM) : max_m;
    L.wmax = (int64_t)align_up((size_t)(cdiv(2 * region_m, 32) > 0 ? cdiv(2 * region_m, 32) : 1),
                               (size_t)8 * kTeam);
    L.region_words = L.wmax + L.wmax / 8;
    L.regions = d->grid_cluster > d->grid_small ? d->grid_cluster : d->grid_small;
    L.lvt_cap = total_n / kVtxTile + G + 1;
    L.lwt_cap = (2 * total_m / 32) / kWordTile + G + 1;
    Carve c;
    L.hdr = c.take(64);
    L.order = c.take((size_t)(G > 0 ? G : 1) * 4);
    L.scratch = c.take((size_t)L.regions * L.region_words * 4);
    L.tabs = c.take((size_t)6 * (G + 1) * 4);
    L.kl = c.take((size_t)L.lvt_cap * kVtxTile * 4);
    L.lbm = c.take((size_t)L.lwt_cap * kWordTile * 4);
    L.lgrp = c.take((size_t)L.lwt_cap * kWordTile / 8 * 4);
    L.lts_scan = c.take((size_t)L.lwt_cap * 8);
    L.lts_emit = c.take((size_t)L.lvt_cap * 8);
    L.total = c.off;
    return true;
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" size_t boba_reorder_batched_workspace_bytes(int64_t G, int64_t max_m, int64_t max_n,
                                                       int64_t total_m, int64_t total_n)
{
    BatchLayout L;
    if (!batch_layout(G, max_m, max_n, total_m, total_n, batch_device(), batch_mode(total_m), L))
        return 0;
    return L.total;
}

extern "C" boba_status_t boba_reorder_batched(const int32_t *src, const int32_t *dst,
                                              const int64_t *edge_off, const int64_t *vert_off,
                                              int64_t G, int64_t max_m, int64_t max_n,
                                              int64_t total_m, int64_t total_n, int32_t *perm_out,
                                              int32_t *src_out, int32_t *dst_out, void *ws,
                                              size_t ws_bytes, void *stream_)
{
    if (G < 0 || max_m < 0 || max_n < 0 || total_m < 0 || total_n < 0) return BOBA_ERR_INVALID_ARG;
    if (max_m > kMaxSize || max_n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    const int mode = batch_mode(total_m);
    if (mode == kBatchCluster && max_n > (int64_t)kTeam * kKcap) return BOBA_ERR_TOO_LARGE;
    if (G == 0) return BOBA_OK;
    if (edge_off == nullptr || vert_off == nullptr) return BOBA_ERR_INVALID_ARG;
    if (total_m > 0 && (src == nullptr || dst == nullptr || src_out == nullptr || dst_out == nullptr))
        return BOBA_ERR_INVALID_ARG;
    if (total_n > 0 && perm_out == nullptr) return BOBA_ERR_INVALID_ARG;
    const BatchDevice *bd = batch_device();
    if (!bd) return BOBA_ERR_CUDA;
    BatchLayout L;
    if (!batch_layout(G, max_m, max_n, total_m, total_n, bd, mode, L)) return BOBA_ERR_INVALID_ARG;
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.dst = dst;
    a.eoff = edge_off;
    a.voff = vert_off;
    a.G = G;
    a.max_m = max_m;
    a.max_n = max_n;
    a.total_m = total_m;
    a.total_n = total_n;
    a.perm = perm_out;
    a.so = src_out;
    a.dout = dst_out;
    a.hdr = reinterpret_cast<uint32_t *>(b + L.hdr);
    a.order = reinterpret_cast<uint32_t *>(b + L.order);
    a.scratch = reinterpret_cast<uint32_t *>(b + L.scratch);
    a.region_words = L.region_words;
    a.wmax = L.wmax;
    a.status = dev->status;
    a.large_threshold = kKcap;
    a.small_max_m = mode == kBatchSplit ? kSmallMaxM : INT64_MAX;
    a.n_limit = mode == kBatchSplit ? kMaxSize : (int64_t)kTeam * kKcap;
    if (mode == kBatchSplit) {
        uint32_t *tabs = reinterpret_cast<uint32_t *>(b + L.tabs);
        a.lg_pc = tabs;
        a.lg_vt = tabs + (G + 1);
        a.lg_wt = tabs + 2 * (G + 1);
        a.lg_ec = tabs + 3 * (G + 1);
        a.lg_tot = tabs + 4 * (G + 1);
        a.lg_st = tabs + 5 * (G + 1);
        a.kl = reinterpret_cast<uint32_t *>(b + L.kl);
        a.lbm = reinterpret_cast<uint32_t *>(b + L.lbm);
        a.lgrp = reinterpret_cast<uint32_t *>(b + L.lgrp);
        a.lts_scan = reinterpret_cast<uint64_t *>(b + L.lts_scan);
        a.lts_emit = reinterpret_cast<uint64_t *>(b + L.lts_emit);
        a.lts_scan_cap = L.lwt_cap;
        a.lts_emit_cap = L.lvt_cap;
        batch_slices(total_m, a.first_smax, a.relabel_smax, a.first_runs, a.relabel_runs);
    }
    BOBA_TIMED("batch.plan", stream, k_batch_plan<<<1, 1024, 0, stream>>>(a));
    if (mode == kBatchCluster) {
        BOBA_TIMED("batch.reorder", stream,
                   k_batch<<<bd->grid_cluster, kBB, kDynSmem, stream>>>(a));
    } else {
        const int gl = bd->sms * 8;
        BOBA_TIMED("batch.small", stream,
                   k_batch_small<<<bd->grid_small, kBB, kDynSmem, stream>>>(a));
        BOBA_TIMED("batch.large.init", stream, k_bl_init<<<gl, kLB, 0, stream>>>(a));
        // graphs of up to fs (rs) slices: sliced kernels; the rest: global ones
        if (a.first_smax > 0)
            BOBA_TIMED("batch.large.first", stream,
                       k_bl_first_sliced<<<bd->grid_small, kBB, kDynSmem, stream>>>(a));
        if (max_n > (int64_t)a.first_smax * kKcap) {
            if (a.first_runs)
                BOBA_TIMED("batch.large.first", stream,
                           k_bl_first_runs<<<bd->sms, kRunBlock, 0, stream>>>(a));
            else
                BOBA_TIMED("batch.large.first", stream, k_bl_first<<<gl, kLB, 0, stream>>>(a));
        }
        BOBA_TIMED("batch.large.mark", stream, k_bl_mark<<<gl, kLB, 0, stream>>>(a));
        BOBA_TIMED("batch.large.scan", stream, k_bl_scan<<<gl, kLB, 0, stream>>>(a));
        BOBA_TIMED("batch.large.emit", stream, k_bl_emit<<<gl, kLB, 0, stream>>>(a));
        if (a.relabel_smax > 0)
            BOBA_TIMED("batch.large.relabel", stream,
                       k_bl_relabel_sliced<<<bd->grid_small, kBB, kDynSmem, stream>>>(a));
        if (max_n > (int64_t)a.relabel_smax * kKcap) {
            if (a.relabel_runs)
                BOBA_TIMED("batch.large.relabel", stream,
                           k_bl_relabel_runs<<<bd->sms, kRunBlock, 0, stream>>>(a));
            else
                BOBA_TIMED("batch.large.relabel", stream, k_bl_relabel<<<gl, kLB, 0, stream>>>(a));
        }
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

// Selects the batched schedule explicitly: 0 cluster, 1 .. 8 split with the
// large-graph phases as batch_slices lists, -1 default.
extern "C" void boba_batched_set_mode(int mode)
{
    g_mode_override = (mode >= 0 && mode <= 8) ? mode : -1;
}
