// PageRank on the pull CSR, the PR application of Sec. 5.1 (arXiv 2306.10410):
// the graph is swept repeatedly until the ranks stop changing.  The paper fixes
// no constants; this is the standard power iteration (Page, Brin, Motwani,
// Winograd 1999) with damping d and the mass of vertices without out-edges
// (dangling vertices) spread uniformly:
//   pr_0(v)     = 1/n
//   D_t         = sum of pr_t(u) over dangling u
//   pr_{t+1}(v) = (1 - d)/n + d * ( (A pr_t)(v) + D_t/n )
// with A the CSR of boba_coo_to_csr (A(v,u) = 1/outdeg(u) per edge u -> v).
//
// The paper's PR pushes each source's share to its neighbours with atomics;
// here it is pulled through the merge-path SpMV, so every step is
// deterministic and needs no floating-point atomics.  Per step:
//   merge-path multiply  y = A pr_t             (spmv.cu; skipped once done)
//   k_pr_update          pr_{t+1} in place, the L1 change and the dangling mass
//                        of pr_{t+1} as per-tile fp64 partials; the last tile
//                        to finish (a ticket) sums the partials in tile order
//                        and sets the next step's constant and the done flag.
// All steps are enqueued up front; after convergence they return at once, so
// the call never waits on the host and can be captured in a CUDA graph.
#include "common.cuh"
#include "host.hpp"

namespace boba {
namespace {

constexpr int kPrBlock = 256;
constexpr int kPrTile = 4096;              // vertices per update block
constexpr int64_t kMaxIters = 1 << 20;

struct PrState {
    double base;          // (1 - d)/n + d * D_t / n for the next update
    double residual;      // L1 change of the last step
    double dangling;      // D of the current iterate
    uint32_t done;        // nonzero: converged, or the input was rejected
    uint32_t ticket;      // tiles of the current update that have finished
    int32_t iters;        // steps taken
    uint32_t bad;         // a column ID outside [0, n)
};

struct PrLayout {
    int64_t mp_tiles, pr_tiles;
    size_t y, has_out, part, state, mp_part, mp_crow, mp_cval, total;
};

bool pr_layout(int64_t n, int64_t nnz, PrLayout &L)
{
    if (n < 0 || nnz < 0 || n > kMaxSize || nnz > kMaxSize) return false;
    L.mp_tiles = cdiv(n + nnz, 2048);              // the smallest tile of any merge-path shape
    L.pr_tiles = cdiv(n, kPrTile);
    Carve c;
    L.y = c.take((size_t)(n > 0 ? n : 1) * 4);
    L.has_out = c.take((size_t)(cdiv(n, 32) + 1) * 4);
    L.part = c.take((size_t)(L.pr_tiles + 1) * 16);
    L.state = c.take(sizeof(PrState));
    L.mp_part = c.take((size_t)(L.mp_tiles + 1) * 8);
    L.mp_crow = c.take((size_t)(L.mp_tiles + 1) * 4);
    L.mp_cval = c.take((size_t)(L.mp_tiles + 1) * 4);
    L.total = c.off;
    return true;
}

// has_out bit u = 1 iff u is a column of some entry, i.e. u has an out-edge.
// Columns below kHubCols (after BOBA, the vertices met first: the busiest
// columns) are collected in a per-block shared bitmap and merged once per
// block, so the hot words are not hammered in L2; the others are set with a
// global atomic after a check that the bit is still clear.
constexpr int kHubCols = 65536;
constexpr int kMarkBlock = 512;

__global__ void __launch_bounds__(kMarkBlock) k_pr_mark(const int32_t *__restrict__ col,
                                                        int64_t nnz, int64_t n, uint32_t *has_out,
                                                        PrState *st, uint32_t *status)
{
    __shared__ uint32_t s_bits[kHubCols / 32];
    const int hub_words = (int)((n < kHubCols ? n : kHubCols) + 31) / 32;
    for (int i = threadIdx.x; i < hub_words; i += kMarkBlock) s_bits[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kMarkBlock;
    for (int64_t j = (int64_t)blockIdx.x * kMarkBlock + threadIdx.x; j < nnz; j += stride) {
        const int32_t u = __ldcs(col + j);
        if (u < 0 || (int64_t)u >= n) {
            raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
            st->bad = 1;
            continue;
        }
        const uint32_t bit = 1u << (u & 31);
        if (u < kHubCols) {
            if ((s_bits[u >> 5] & bit) == 0) atomicOr(&s_bits[u >> 5], bit);
        } else if ((__ldcg(has_out + (u >> 5)) & bit) == 0) {
            atomicOr(has_out + (u >> 5), bit);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < hub_words; i += kMarkBlock) {
        const uint32_t w = s_bits[i];
        if (w != 0 && (__ldcg(has_out + i) & w) != w) atomicOr(has_out + i, w);
    }
}

// Sum of a double over the block in a fixed order (xor tree in each warp, then
// the warps' sums in warp order).  The result is valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double *s_warp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kPrBlock / 32; ++w) t += s_warp[w];
    return t;
}

// INIT: pr = 1/n and the dangling mass of pr_0.  Otherwise one step:
// pr(v) <- base + d * y(v), with the step's L1 change.
template <bool INIT>
__global__ void __launch_bounds__(kPrBlock) k_pr_update(
    float *__restrict__ pr, const float *__restrict__ y, const uint32_t *__restrict__ has_out,
    int64_t n, double d, double tol, int64_t max_iters, PrState *st, double2 *part,
    int32_t *iters_out, double *residual_out)
{
    __shared__ double s_warp[kPrBlock / 32];
    __shared__ bool s_last;
    if (!INIT && *(volatile uint32_t *)&st->done) return;
    const float df = (float)d;
    const float base = INIT ? 0.0f : (float)st->base;
    const float inv_n = (float)(1.0 / (double)n);
    // a thread's 16 terms are summed in fp32 (relative error below 1e-6), the
    // block and tile sums in fp64: few fp64 operations, which are slow here
    float change = 0.0f, dangling = 0.0f;
    const int64_t v0 = (int64_t)blockIdx.x * kPrTile;
    for (int k = threadIdx.x; k < kPrTile; k += kPrBlock) {
        const int64_t v = v0 + k;
        if (v >= n) break;
        float nv;
        if (INIT) {
            nv = inv_n;
        } else {
            const float old = pr[v];
            nv = fmaf(df, __ldcs(y + v), base);
            change += fabsf(nv - old);
        }
        pr[v] = nv;
        if (((__ldg(has_out + (v >> 5)) >> (v & 31)) & 1u) == 0) dangling += nv;
    }
    const double c = block_sum_fixed((double)change, s_warp);
    const double g = block_sum_fixed((double)dangling, s_warp);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = make_double2(c, g);
        __threadfence();
        s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last tile: every partial is visible (each was fenced before its ticket)
    __threadfence();
    double cs = 0.0, gs = 0.0;
    for (int64_t t = threadIdx.x; t < (int64_t)gridDim.x; t += kPrBlock) {
        const double2 p = __ldcg(part + t);
        cs += p.x;
        gs += p.y;
    }
    // a fixed-shape tree over the threads' strided sums
    const double C = block_sum_fixed(cs, s_warp);
    const double G = block_sum_fixed(gs, s_warp);
    if (threadIdx.x == 0) {
        st->ticket = 0;
        st->dangling = G;
        st->base = (1.0 - d) / (double)n + d * G / (double)n;
        if (INIT) {
            st->iters = 0;
            st->residual = 0.0;
            st->done = (st->bad != 0 || max_iters == 0) ? 1u : 0u;
        } else {
            st->iters += 1;
            st->residual = C;
            if (C < tol) st->done = 1;
        }
        if (iters_out) *iters_out = st->iters;
        if (residual_out) *residual_out = st->residual;
    }
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" size_t boba_pagerank_workspace_bytes(int64_t n, int64_t nnz)
{
    PrLayout L;
    if (!pr_layout(n, nnz, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_pagerank(const int64_t *row_ptr, const int32_t *col,
                                       const float *val, int64_t n, int64_t nnz, double damping,
                                       int64_t max_iters, double tol, float *pr,
                                       int32_t *iters_out, double *residual_out, void *ws,
                                       size_t ws_bytes, void *stream_)
{
    if (n < 0 || nnz < 0 || max_iters < 0 || max_iters > kMaxIters) return BOBA_ERR_INVALID_ARG;
    if (!(damping >= 0.0 && damping < 1.0) || !(tol >= 0.0)) return BOBA_ERR_INVALID_ARG;
    if (n > kMaxSize || nnz > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && nnz > 0) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (row_ptr == nullptr || pr == nullptr) return BOBA_ERR_INVALID_ARG;
    if (nnz > 0 && (col == nullptr || val == nullptr)) return BOBA_ERR_INVALID_ARG;
    PrLayout L;
    pr_layout(n, nnz, L);
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    float *y = reinterpret_cast<float *>(b + L.y);
    uint32_t *has_out = reinterpret_cast<uint32_t *>(b + L.has_out);
    double2 *part = reinterpret_cast<double2 *>(b + L.part);
    PrState *st = reinterpret_cast<PrState *>(b + L.state);
    int2 *mp_part = reinterpret_cast<int2 *>(b + L.mp_part);
    int32_t *crow = reinterpret_cast<int32_t *>(b + L.mp_crow);
    float *cval = reinterpret_cast<float *>(b + L.mp_cval);

    BOBA_CUDA_TRY(cudaMemsetAsync(has_out, 0, (size_t)(cdiv(n, 32) + 1) * 4, s));
    BOBA_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(PrState), s));
    if (nnz > 0) {
        const int g = persistent_grid((const void *)k_pr_mark, kMarkBlock, cdiv(nnz, kMarkBlock));
        BOBA_TIMED("pagerank.mark", s,
                   k_pr_mark<<<g, kMarkBlock, 0, s>>>(col, nnz, n, has_out, st, dev->status));
    }
    const unsigned tiles = (unsigned)L.pr_tiles;
    BOBA_TIMED("pagerank.update", s,
               k_pr_update<true><<<tiles, kPrBlock, 0, s>>>(pr, nullptr, has_out, n, damping, tol,
                                                            max_iters, st, part, iters_out,
                                                            residual_out));
    int variant = tuned_variant(kTuneSpmv, nnz);
    if (variant < 5 || variant > 14) variant = 5;
    if (max_iters > 0)
        merge_path_partition(row_ptr, n, nnz, merge_path_items(variant), mp_part, s);
    for (int64_t t = 0; t < max_iters; ++t) {
        merge_path_multiply(variant, row_ptr, col, val, pr, y, n, nnz, mp_part, crow, cval,
                            &st->done, s);
        BOBA_TIMED("pagerank.update", s,
                   k_pr_update<false><<<tiles, kPrBlock, 0, s>>>(pr, y, has_out, n, damping, tol,
                                                                 max_iters, st, part, iters_out,
                                                                 residual_out));
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
