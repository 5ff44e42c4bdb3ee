// Batched BOBA: G independent graphs of uneven sizes in one persistent launch
// (arXiv 2306.10410, Alg. 2 with AtomicMin, per graph).
//
// Each graph is processed whole by one team of CTAs, so no CTA ever waits on
// another outside a hardware cluster barrier:
//   * a graph with at most kKcap vertices is handled by a single CTA; its keys
//     and then its labels live in that CTA's shared memory;
//   * a larger graph (up to kTeam * kKcap vertices) is handled by a cluster of
//     kTeam CTAs; its vertex range is split evenly and each CTA keeps its
//     slice of the key/label array in its shared memory, which the other CTAs
//     of the cluster reach through distributed shared memory.
// Per graph the team runs the same steps as the single-graph path: keys =
// SENT, first occurrence (atomicMin into shared memory), first-occurrence
// bitmap (global scratch, resident in L2), its popcount prefix, labels (rank
// of the key; vertices on no edge after them by ascending ID) written over the
// keys in place, and the relabel of both endpoint arrays.
//
// k_batch_plan orders the work: large graphs first, then small graphs in packs
// of kTeam (one per CTA of a cluster), each class by decreasing edge count in
// power-of-two buckets, so that the longest items start first.
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"
#include "host.hpp"

namespace cg = cooperative_groups;

namespace boba {
namespace {

constexpr int kBB = 1024;                  // threads per CTA
constexpr int kTeam = 8;                   // CTAs per cluster, team size for large graphs
constexpr int kKcap = 54 * 1024;           // vertices per CTA held in shared memory
constexpr size_t kDynSmem = (size_t)kKcap * 4;
constexpr int kU = 8;                      // stream loads in flight per thread
constexpr int kHdrItems = 0, kHdrLarge = 1, kHdrTicket = 2, kHdrValid = 3;

struct BatchArgs {
    const int32_t *src, *dst;
    const int64_t *eoff, *voff;
    int64_t G, max_m, max_n, total_m, total_n;
    int32_t *perm, *so, *dout;
    uint32_t *hdr;           // items, large graphs, ticket, valid graphs
    uint32_t *order;         // graph ids in processing order
    uint32_t *scratch;       // one region per CTA of the grid
    int64_t region_words;    // wmax bitmap words + wmax/8 group-prefix words
    int64_t wmax;
    uint32_t *status;
};

__device__ __forceinline__ int floor_log2_p1(int64_t x)   // floor(log2(x + 1)), x >= 0
{
    return 63 - __clzll((unsigned long long)(x + 1));
}

// One block of 1024 threads: validate the offsets, bucket the graphs, write
// the processing order and the work header, reset the ticket.
__global__ void __launch_bounds__(1024) k_batch_plan(BatchArgs a)
{
    __shared__ uint32_t hist[128], cur[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t g = threadIdx.x; g < a.G; g += blockDim.x) {
        const int64_t e0 = a.eoff[g], e1 = a.eoff[g + 1], v0 = a.voff[g], v1 = a.voff[g + 1];
        const int64_t m = e1 - e0, n = v1 - v0;
        const bool ok = e0 >= 0 && v0 >= 0 && m >= 0 && n >= 0 && e1 <= a.total_m &&
                        v1 <= a.total_n && m <= a.max_m && n <= a.max_n &&
                        n <= (int64_t)kTeam * kKcap && !(n == 0 && m > 0);
        if (!ok) { raise_status(a.status, BOBA_ERR_INVALID_ARG); continue; }
        if (n == 0) continue;
        const int lg = floor_log2_p1(m) & 63;
        const int b = (n > kKcap ? 0 : 64) + (63 - lg);
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
    }
    __syncthreads();
    for (int64_t g = threadIdx.x; g < a.G; g += blockDim.x) {
        const int64_t e0 = a.eoff[g], e1 = a.eoff[g + 1], v0 = a.voff[g], v1 = a.voff[g + 1];
        const int64_t m = e1 - e0, n = v1 - v0;
        const bool ok = e0 >= 0 && v0 >= 0 && m >= 0 && n >= 0 && e1 <= a.total_m &&
                        v1 <= a.total_n && m <= a.max_m && n <= a.max_n &&
                        n <= (int64_t)kTeam * kKcap && !(n == 0 && m > 0);
        if (!ok || n == 0) continue;
        const int lg = floor_log2_p1(m) & 63;
        const int b = (n > kKcap ? 0 : 64) + (63 - lg);
        a.order[atomicAdd(&cur[b], 1u)] = (uint32_t)g;
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
__device__ __forceinline__ void team_sync(cg::cluster_group &cl)
{
    if constexpr (T == 1) __syncthreads();
    else cl.sync();
}

template <int T>
__device__ __forceinline__ uint32_t *key_ptr(uint32_t *s_keys, TeamSmem &ts, uint32_t owner)
{
    if constexpr (T == 1) return s_keys;
    else return ts.kp[owner];
}

// Process graph g with a team of T CTAs; this CTA is member t, the team's CTAs
// are grid CTAs cta0 .. cta0+T-1 (their scratch regions).
template <int T>
__device__ void process_graph(const BatchArgs &a, uint32_t g, int t, int64_t cta0,
                              cg::cluster_group &cl, uint32_t *s_keys, TeamSmem &ts)
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
        if (tid < T) ts.kp[tid] = cl.map_shared_rank(s_keys, tid);
    }
    // 1. keys = SENT, clear this member's bitmap slice
    for (int64_t i = tid; i < myn; i += kBB) s_keys[i] = kSent;
    for (int64_t w = tid; w < Wc; w += kBB) my_bm[w] = 0u;
    team_sync<T>(cl);

    // 2. first occurrence over this member's share of I ++ J: kU loads in
    // flight per thread, then all key reads, then the (rare) atomics
    {
        const int64_t P = 2 * m;
        const int64_t lo = P * t / T, hi = P * (t + 1) / T;
        for (int64_t b0 = lo + tid; b0 < hi; b0 += (int64_t)kU * kBB) {
            int32_t v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t i = b0 + (int64_t)u * kBB;
                v[u] = -1;
                if (i < hi) v[u] = i < m ? __ldcs(a.src + E0 + i) : __ldcs(a.dst + E0 + (i - m));
            }
            uint32_t own[kU], li[kU], cur[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t i = b0 + (int64_t)u * kBB;
                own[u] = kTeam;                                  // "skip"
                li[u] = 0;
                cur[u] = 0;
                if (i < hi) {
                    if ((uint32_t)v[u] < nn) {
                        own[u] = (uint32_t)v[u] / chunk;
                        li[u] = (uint32_t)v[u] - own[u] * chunk;
                        cur[u] = key_ptr<T>(s_keys, ts, own[u])[li[u]];
                    } else {
                        raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t i = (uint32_t)(b0 + (int64_t)u * kBB);
                if (own[u] < kTeam && cur[u] > i) atomicMin(key_ptr<T>(s_keys, ts, own[u]) + li[u], i);
            }
        }
    }
    team_sync<T>(cl);

    // 3. mark first-occurrence positions; count vertices on no edge
    uint32_t iso = 0;
    for (int64_t i = tid; i < myn; i += kBB) {
        const uint32_t k = s_keys[i];
        if (k == kSent) { ++iso; continue; }
        const int64_t w = k >> 5;
        const int64_t r = w / Wc;
        atomicOr(a.scratch + (cta0 + r) * a.region_words + (w - r * Wc), 1u << (k & 31u));
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
                tr = *cl.map_shared_rank(&ts.xtot, r);
                ir = *cl.map_shared_rank(&ts.xiso, r);
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
                    const int64_t w = k >> 5;
                    const int64_t r = w / Wc;
                    const int64_t wl = w - r * Wc;
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
        const int64_t lo = m * t / T, hi = m * (t + 1) / T;
        for (int64_t b0 = lo + tid; b0 < hi; b0 += (int64_t)U2 * kBB) {
            int32_t v[kU];
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const int64_t e = b0 + (int64_t)u * kBB;
                v[2 * u] = v[2 * u + 1] = -1;
                if (e < hi) {
                    v[2 * u] = __ldcs(a.src + E0 + e);
                    v[2 * u + 1] = __ldcs(a.dst + E0 + e);
                }
            }
            int32_t lab[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                lab[u] = -1;
                if ((uint32_t)v[u] < nn) {
                    const uint32_t o = (uint32_t)v[u] / chunk;
                    lab[u] = (int32_t)key_ptr<T>(s_keys, ts, o)[(uint32_t)v[u] - o * chunk];
                }
            }
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const int64_t e = b0 + (int64_t)u * kBB;
                if (e >= hi) continue;
                if (lab[2 * u] < 0 || lab[2 * u + 1] < 0)
                    raise_status(a.status, BOBA_ERR_ID_OUT_OF_RANGE);
                __stcs(a.so + E0 + e, lab[2 * u]);
                __stcs(a.dout + E0 + e, lab[2 * u + 1]);
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
            process_graph<kTeam>(a, a.order[item], rank, cluster_cta0, cl, s_keys, ts);
        } else {
            const uint32_t idx = n_large + (item - n_large) * kTeam + (uint32_t)rank;
            if (idx < a.hdr[kHdrValid])
                process_graph<1>(a, a.order[idx], 0, (int64_t)blockIdx.x, cl, s_keys, ts);
        }
    }
}

struct BatchDevice {
    bool ready = false;
    int grid_ctas = 0;
};
std::mutex g_bmu;
BatchDevice g_bdev[64];

// Grid of the persistent launch on the current device: every cluster that fits.
int batch_grid_ctas()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchDevice &d = g_bdev[dev];
    if (!d.ready) {
        if (cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDynSmem) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kTeam, 1, 1);
        cfg.blockDim = dim3(kBB, 1, 1);
        cfg.dynamicSmemBytes = kDynSmem;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)k_batch, &cfg) != cudaSuccess ||
            clusters < 1) {
            (void)cudaGetLastError();
            return 0;
        }
        d.grid_ctas = clusters * kTeam;
        d.ready = true;
    }
    return d.grid_ctas;
}

struct BatchLayout {
    int64_t wmax, region_words;
    size_t hdr, order, scratch, total;
};

bool batch_layout(int64_t G, int64_t max_m, int64_t max_n, int grid_ctas, BatchLayout &L)
{
    if (G < 0 || max_m < 0 || max_n < 0 || max_m > kMaxSize || max_n > kMaxSize || grid_ctas < 1)
        return false;
    L.wmax = (int64_t)align_up((size_t)(cdiv(2 * max_m, 32) > 0 ? cdiv(2 * max_m, 32) : 1),
                               (size_t)8 * kTeam);
    L.region_words = L.wmax + L.wmax / 8;
    Carve c;
    L.hdr = c.take(64);
    L.order = c.take((size_t)(G > 0 ? G : 1) * 4);
    L.scratch = c.take((size_t)grid_ctas * L.region_words * 4);
    L.total = c.off;
    return true;
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" size_t boba_reorder_batched_workspace_bytes(int64_t G, int64_t max_m, int64_t max_n)
{
    BatchLayout L;
    if (!batch_layout(G, max_m, max_n, batch_grid_ctas(), L)) return 0;
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
    if (max_n > (int64_t)kTeam * kKcap) return BOBA_ERR_TOO_LARGE;
    if (G == 0) return BOBA_OK;
    if (edge_off == nullptr || vert_off == nullptr) return BOBA_ERR_INVALID_ARG;
    if (total_m > 0 && (src == nullptr || dst == nullptr || src_out == nullptr || dst_out == nullptr))
        return BOBA_ERR_INVALID_ARG;
    if (total_n > 0 && perm_out == nullptr) return BOBA_ERR_INVALID_ARG;
    const int grid = batch_grid_ctas();
    if (grid < 1) return BOBA_ERR_CUDA;
    BatchLayout L;
    if (!batch_layout(G, max_m, max_n, grid, L)) return BOBA_ERR_INVALID_ARG;
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    BatchArgs a;
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
    BOBA_TIMED("batch.plan", stream, k_batch_plan<<<1, 1024, 0, stream>>>(a));
    BOBA_TIMED("batch.reorder", stream, k_batch<<<grid, kBB, kDynSmem, stream>>>(a));
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
