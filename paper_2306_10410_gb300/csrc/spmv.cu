// Pull SpMV, Alg. 3 (arXiv 2306.10410, Sec. 1.2.2): y(v) = sum over the
// entries of row v of A(v,u) * x(u), fp32 products and fp32 accumulation.
//
//   k_spmv_rows    groups of LPR lanes per row (LPR = 32 is warp-per-row; for a
//                  short average row length several rows share a warp).  Lane j
//                  of a group sums entries j, j+LPR, ... with FMA; the group then
//                  reduces with a fixed xor tree.  Rows longer than kLongRow are
//                  set aside in a list.
//   k_spmv_plan    one block: chunk offsets of the long rows (kChunk entries each)
//   k_spmv_chunks  one 1024-thread block per chunk: strided FMA sums and a
//                  fixed-order block reduction into partial[chunk]
//   k_spmv_gather  y[long row] = its chunk partials summed in chunk order
// Every summation order depends only on the row's own entries (and on LPR, a
// function of nnz / n_rows), so the result is the same on every run, and rows of
// equal content give equal bits whatever their index.
//
//   k_mp_partition / k_mp_spmv / k_mp_fixup   the merge-path SpMV (below),
//                  the tuned choice for skewed graphs; its shapes differ in
//                  block size, items per thread and shared-memory carve-out.
#include <atomic>

#include "common.cuh"
#include "host.hpp"

namespace boba {
namespace {

constexpr int64_t kLongRow = 4096;     // entries; longer rows are chunked
constexpr int64_t kChunk = 16384;      // entries per chunk of a long row
constexpr int kChunkBlock = 1024;
constexpr int kRowsBlock = 256;

constexpr int kMpTile = 2048;      // smallest merge-path tile (path items) of any shape

struct SpmvLayout {
    int64_t cap, max_chunks, mp_tiles;
    size_t count, list, cstart, partial, mp_part, mp_crow, mp_cval, total;
};

bool spmv_layout(int64_t n_rows, int64_t nnz, SpmvLayout &L)
{
    if (n_rows < 0 || nnz < 0 || n_rows > kMaxSize || nnz > kMaxSize) return false;
    L.cap = nnz / kLongRow + 1;
    L.max_chunks = nnz / kChunk + L.cap + 1;
    Carve c;
    L.count = c.take(64);
    L.list = c.take((size_t)L.cap * 4);
    L.cstart = c.take((size_t)(L.cap + 1) * 4);
    L.partial = c.take((size_t)L.max_chunks * 4);
    L.mp_tiles = cdiv(n_rows + nnz, kMpTile);
    L.mp_part = c.take((size_t)(L.mp_tiles + 1) * 8);
    L.mp_crow = c.take((size_t)(L.mp_tiles + 1) * 4);
    L.mp_cval = c.take((size_t)(L.mp_tiles + 1) * 4);
    L.total = c.off;
    return true;
}

template <int LPR>
__global__ void __launch_bounds__(kRowsBlock) k_spmv_rows(
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y,
    int64_t n_rows, uint32_t *long_count, uint32_t *long_list, uint32_t cap, uint32_t *status)
{
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int gl = lane % LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t rb = warp * RPW; rb < n_rows; rb += nwarps * RPW) {
        const int64_t r = rb + lane / LPR;
        int64_t beg = 0, end = 0;
        if (r < n_rows) {
            beg = __ldg(row_ptr + r);
            end = __ldg(row_ptr + r + 1);
        }
        const bool is_long = end - beg > kLongRow;
        float acc = 0.0f;
        if (!is_long) {
#pragma unroll 4
            for (int64_t p = beg + gl; p < end; p += LPR)
                acc = fmaf(__ldcs(val + p), __ldg(x + __ldcs(col + p)), acc);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (gl == 0 && r < n_rows) {
            if (!is_long) {
                y[r] = acc;
            } else {
                const uint32_t i = atomicAdd(long_count, 1u);
                if (i < cap) long_list[i] = (uint32_t)r;
                else raise_status(status, BOBA_ERR_INVALID_ARG);   // row_ptr inconsistent with nnz
            }
        }
    }
}

// Chunk offsets of the long rows: cstart[i] = sum over j < i of ceil(len_j / kChunk).
__global__ void __launch_bounds__(256) k_spmv_plan(const int64_t *__restrict__ row_ptr,
                                                   const uint32_t *long_count,
                                                   const uint32_t *__restrict__ long_list,
                                                   uint32_t cap, uint32_t *cstart)
{
    __shared__ typename BlockScan<256>::Smem sm;
    const uint32_t L = min(*long_count, cap);
    uint32_t carry = 0;
    for (uint32_t base = 0; base < L; base += 256) {
        const uint32_t i = base + threadIdx.x;
        uint32_t c = 0;
        if (i < L) {
            const uint32_t r = long_list[i];
            c = (uint32_t)cdiv(row_ptr[r + 1] - row_ptr[r], kChunk);
        }
        uint32_t tot;
        const uint32_t ex = BlockScan<256>::exclusive(c, &tot, sm);
        if (i < L) cstart[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) cstart[L] = carry;
}

__global__ void __launch_bounds__(kChunkBlock) k_spmv_chunks(
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, const uint32_t *long_count,
    const uint32_t *__restrict__ long_list, uint32_t cap, const uint32_t *__restrict__ cstart,
    float *__restrict__ partial)
{
    __shared__ float s_w[kChunkBlock / 32];
    const uint32_t L = min(*long_count, cap);
    const uint32_t C = cstart[L];
    for (uint32_t c = blockIdx.x; c < C; c += gridDim.x) {
        // the long row owning chunk c: last i with cstart[i] <= c
        uint32_t lo = 0, hi = L;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cstart[mid] <= c) lo = mid; else hi = mid;
        }
        const uint32_t r = long_list[lo];
        const int64_t beg = row_ptr[r] + (int64_t)(c - cstart[lo]) * kChunk;
        const int64_t end = min(row_ptr[r + 1], beg + kChunk);
        float acc = 0.0f;
#pragma unroll 4
        for (int64_t p = beg + threadIdx.x; p < end; p += kChunkBlock)
            acc = fmaf(__ldcs(val + p), __ldg(x + __ldcs(col + p)), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            float w = s_w[threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            if (threadIdx.x == 0) partial[c] = w;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_spmv_gather(const uint32_t *long_count,
                                                     const uint32_t *__restrict__ long_list,
                                                     uint32_t cap, const uint32_t *__restrict__ cstart,
                                                     const float *__restrict__ partial,
                                                     float *__restrict__ y)
{
    const uint32_t L = min(*long_count, cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (uint32_t c = cstart[i]; c < cstart[i + 1]; ++c) s += partial[c];
        y[long_list[i]] = s;
    }
}

// ---------------------------------------------------------------------------
// Merge-path SpMV (Merrill and Garland, "Merge-based parallel sparse matrix-
// vector multiplication", SC 2016), the load balancing of the paper's
// evaluation (Sec. 3.3 and 5.1): the path of n_rows row ends and nnz nonzeros is
// cut into tiles of block x items path items (the shapes of kMpShapes), so
// every block gets the same work whatever the row lengths.  Sums run in path order within a thread, then a segmented scan
// over the threads of a tile, then (for rows crossing tiles) the tiles'
// carries in tile order: deterministic, but the rounding depends on where a
// row falls relative to the tiles.
// ---------------------------------------------------------------------------

// Split of diagonal d of the merge of row_ptr[1..n] with 0..nnz-1: x row ends
// and y nonzeros lie before it (x + y = d).
__device__ __forceinline__ void mp_search(const int64_t *__restrict__ row_ptr, int64_t n,
                                          int64_t nnz, int64_t d, int64_t &x, int64_t &y)
{
    int64_t lo = d - nnz > 0 ? d - nnz : 0, hi = d < n ? d : n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(row_ptr + mid + 1) <= d - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    x = lo;
    y = d - lo;
}

__global__ void __launch_bounds__(256) k_mp_partition(const int64_t *__restrict__ row_ptr, int64_t n,
                                                      int64_t nnz, int64_t tiles, int64_t tile_items,
                                                      int2 *part)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const int64_t d = t * tile_items < n + nnz ? t * tile_items : n + nnz;
    int64_t x, y;
    mp_search(row_ptr, n, nnz, d, x, y);
    part[t] = make_int2((int)x, (int)y);
}

struct KV {
    int32_t k;
    float v;
};

// The shared arrays of one merge-path tile, padded one word per 32 (a thread
// walks MI consecutive items, so without the padding the lanes of a warp would
// hit the same few banks): the row ends of the tile's rows, then the products
// of its nonzeros, in one buffer -- rows and nonzeros together are the tile's
// MB * MI path items, so one tile's worth of words holds both.  Half the
// shared memory of two separate arrays leaves that much more L1 for the x
// gathers.  And the warp carries.
template <int MB, int MI>
struct MpSmem {
    static constexpr int kWords = MB * MI + MB * MI / 32 + 4;
    int32_t s_buf[kWords];
    KV s_warp[MB / 32];
};

// A gather of x that asks L1 to keep the line (evict-last).  On a BOBA order
// the vertices that appear most often take the smallest labels, so the first
// entries of x are gathered far more often than the rest (R-MAT 24, 2^28
// edges: x[0, 65536) serves 32 % of the nonzeros); marking their lines helps
// them stay in L1 against the one-off lines of the other gathers.
__device__ __forceinline__ float ld_x_keep(const float *p)
{
    float v;
    asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// One tile of the merge path: the tile's rows and nonzeros split evenly over
// the MB threads (MI path items each).  With HOT, columns below `hot` are
// gathered by ld_x_keep.  Both loads are issued by every lane, each lane
// pointing the one it does not need at x[0]: a per-lane branch between two
// loads would serialise them and stall the gathers in flight.
template <int MB, int MI, bool HOT = false>
__device__ __forceinline__ void mp_tile(
    int64_t tile, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y,
    const int2 *__restrict__ part, int32_t *__restrict__ carry_row, float *__restrict__ carry_val,
    MpSmem<MB, MI> &sm, int32_t hot = 0)
{
    constexpr int kMpBlock = MB, kMpItems = MI;
    auto P = [](int j) { return j + (j >> 5); };
    const int2 p0 = part[tile], p1 = part[tile + 1];
    const int x0 = p0.x, y0 = p0.y;
    const int nrows = p1.x - p0.x, nnzt = p1.y - p0.y;
    // row ends at P(0 .. nrows) (the last one a sentinel), products after them
    int32_t *s_end = sm.s_buf;
    float *s_prod = reinterpret_cast<float *>(sm.s_buf + P(nrows) + 1);
    KV *s_warp = sm.s_warp;
    for (int i = threadIdx.x; i < nrows; i += kMpBlock)
        s_end[P(i)] = (int32_t)(__ldg(row_ptr + x0 + 1 + i) - y0);
    if (threadIdx.x == 0) s_end[P(nrows)] = 0x7FFFFFFF;   // sentinel: no row end beyond
#pragma unroll
    for (int u = 0; u < kMpItems; ++u) {
        const int j = u * kMpBlock + threadIdx.x;
        if (j < nnzt) {
            const int32_t c = __ldcs(col + y0 + j);
            float xv;
            if constexpr (HOT) {
                const bool h = c < hot;
                const float a = ld_x_keep(x + (h ? c : 0));
                const float b = __ldg(x + (h ? 0 : c));
                xv = h ? a : b;
            } else {
                xv = __ldg(x + c);
            }
            s_prod[P(j)] = __ldcs(val + y0 + j) * xv;
        }
    }
    __syncthreads();
    // this thread's split inside the tile
    const int dt = threadIdx.x * kMpItems < nrows + nnzt ? threadIdx.x * kMpItems : nrows + nnzt;
    int lo = dt - nnzt > 0 ? dt - nnzt : 0, hi = dt < nrows ? dt : nrows;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[P(mid)] <= dt - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    int xt = lo, yt = dt - lo;
    const int first_row = xt;
    float acc = 0.0f;
    float first_val = 0.0f;         // partial of the first row end this thread consumes
    int first_end = -1;             // that row (relative), or -1 if none
    // consume kMpItems path items in order; the current row's end stays in a
    // register and is reloaded only when the row changes
    int row_end = s_end[P(xt)];
#pragma unroll
    for (int i = 0; i < kMpItems; ++i) {
        if (xt + yt >= nrows + nnzt) break;
        if (yt < row_end) {
            acc += s_prod[P(yt)];
            ++yt;
        } else {
            if (first_end < 0) { first_end = xt; first_val = acc; }
            else y[x0 + xt] = acc;                 // row begun and ended in this thread
            acc = 0.0f;
            ++xt;
            row_end = s_end[P(xt)];
        }
    }
    // segmented scan of the threads' trailing partials (row xt, value acc):
    // carry_in(t) = partial of row first_row accumulated by earlier threads
    KV mine = {xt, acc};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    KV inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t k = __shfl_up_sync(kFull, inc.k, o);
        const float v = __shfl_up_sync(kFull, inc.v, o);
        if (lane >= o && k == inc.k) inc.v = v + inc.v;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        KV w = lane < kMpBlock / 32 ? s_warp[lane] : KV{-1, 0.0f};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t k = __shfl_up_sync(kFull, w.k, o);
            const float v = __shfl_up_sync(kFull, w.v, o);
            if (lane >= o && k == w.k) w.v = v + w.v;
        }
        if (lane < kMpBlock / 32) s_warp[lane] = w;       // inclusive over warps
    }
    __syncthreads();
    if (warp > 0) {
        const KV pw = s_warp[warp - 1];
        if (pw.k == inc.k) inc.v = pw.v + inc.v;
    }
    // carry into this thread: the inclusive value of thread t-1 if it ended on first_row
    KV prev;
    prev.k = __shfl_up_sync(kFull, inc.k, 1);
    prev.v = __shfl_up_sync(kFull, inc.v, 1);
    if (lane == 0) prev = warp > 0 ? s_warp[warp - 1] : KV{-1, 0.0f};
    const float cin = (threadIdx.x > 0 && prev.k == first_row) ? prev.v : 0.0f;
    if (first_end >= 0) y[x0 + first_end] = cin + first_val;
    if (threadIdx.x == kMpBlock - 1) {
        // the tile's trailing partial (row continues into the next tile)
        carry_row[tile] = x0 + inc.k;
        carry_val[tile] = inc.v;
    }
}

// CARVE only makes separate instances, so that a shared-memory carve-out set
// for one variant does not apply to the others.  HOT: see mp_tile.
template <int MB, int MI, int CARVE = 0, bool HOT = false>
__global__ void __launch_bounds__(MB) k_mp_spmv(
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y, int64_t n,
    int64_t nnz, const int2 *__restrict__ part, int32_t *__restrict__ carry_row,
    float *__restrict__ carry_val, const uint32_t *skip, int32_t hot)
{
    if (skip != nullptr && *skip != 0) return;       // an iterative caller has converged
    __shared__ MpSmem<MB, MI> sm;
    mp_tile<MB, MI, HOT>(blockIdx.x, row_ptr, col, val, x, y, part, carry_row, carry_val, sm, hot);
}

// y[r] += the carries of the tiles that ended inside row r, in tile order.
__global__ void __launch_bounds__(256) k_mp_fixup(const int32_t *__restrict__ carry_row,
                                                  const float *__restrict__ carry_val,
                                                  int64_t tiles, int64_t n, float *__restrict__ y,
                                                  const uint32_t *skip)
{
    if (skip != nullptr && *skip != 0) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const int32_t r = carry_row[t];
    if (t > 0 && carry_row[t - 1] == r) return;          // not the first tile of the run
    if (r >= n) return;
    float s = 0.0f;
    for (int64_t u = t; u < tiles && carry_row[u] == r; ++u) s += carry_val[u];
    y[r] = s + y[r];
}

template <int LPR>
void launch_rows(const int64_t *row_ptr, const int32_t *col, const float *val, const float *x,
                 float *y, int64_t n_rows, uint32_t *cnt, uint32_t *list, uint32_t cap,
                 uint32_t *status, cudaStream_t stream)
{
    constexpr int RPW = 32 / LPR;
    const int64_t warps = cdiv(n_rows, RPW);
    const int g = persistent_grid((const void *)k_spmv_rows<LPR>, kRowsBlock,
                                  cdiv(warps, kRowsBlock / 32));
    BOBA_TIMED("spmv", stream,
               k_spmv_rows<LPR><<<g, kRowsBlock, 0, stream>>>(row_ptr, col, val, x, y, n_rows, cnt,
                                                             list, cap, status));
}

}  // namespace

// Merge-path shapes of the tuned SpMV variants 5 .. 14: threads per block,
// path items per thread, the cap on the shared-memory carve-out in KB (0: the
// default, which maximises resident blocks), and the hot prefix of x in
// entries (0: none; see mp_tile).  A smaller carve-out trades resident warps
// for L1, which holds the hot x entries.
struct MpShape {
    int block, items, carve_kb, hot;
};
constexpr MpShape kMpShapes[] = {
    {256, 8, 0, 0}, {256, 12, 0, 0}, {512, 8, 0, 0}, {128, 16, 0, 0},          // 5 .. 8
    {256, 8, 64, 0}, {256, 8, 32, 0}, {256, 12, 64, 0}, {512, 8, 64, 0},       // 9 .. 12
    {256, 16, 64, 0}, {256, 12, 64, 65536},                                    // 13 .. 14
};
constexpr int kMpFirst = 5, kMpLast = 14;

MpShape mp_shape(int variant)
{
    if (variant < kMpFirst || variant > kMpLast) variant = kMpFirst;
    return kMpShapes[variant - kMpFirst];
}

int merge_path_items(int variant)
{
    const MpShape sh = mp_shape(variant);
    return sh.block * sh.items;
}

namespace {

// One launch of k_mp_spmv<MB, MI, CARVE, HOT>; with a carve-out cap the
// attribute is set on that instance only, once per device.
template <int MB, int MI, int CARVE, bool HOT = false>
void launch_mp(int carve_kb, int hot, const int64_t *row_ptr, const int32_t *col,
               const float *val, const float *x, float *y, int64_t n, int64_t nnz,
               const int2 *part, int32_t *crow, float *cval, const uint32_t *skip, int64_t tiles,
               cudaStream_t stream)
{
    static std::atomic<uint64_t> done{0};          // devices whose attribute is set
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (carve_kb > 0 && (done.load() & bit) == 0) {
        cudaFuncSetAttribute((const void *)k_mp_spmv<MB, MI, CARVE, HOT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, carve_kb * 100 / 228);
        done.fetch_or(bit);
    }
    BOBA_TIMED("spmv", stream,
               k_mp_spmv<MB, MI, CARVE, HOT><<<(unsigned)tiles, MB, 0, stream>>>(
                   row_ptr, col, val, x, y, n, nnz, part, crow, cval, skip, (int32_t)hot));
}

}  // namespace

void merge_path_partition(const int64_t *row_ptr, int64_t n, int64_t nnz, int items, int2 *part,
                          cudaStream_t stream)
{
    const int64_t tiles = cdiv(n + nnz, items);
    BOBA_TIMED("spmv.partition", stream,
               k_mp_partition<<<(unsigned)cdiv(tiles + 1, 256), 256, 0, stream>>>(
                   row_ptr, n, nnz, tiles, items, part));
}

void merge_path_multiply(int variant, const int64_t *row_ptr, const int32_t *col, const float *val,
                         const float *x, float *y, int64_t n, int64_t nnz, const int2 *part,
                         int32_t *crow, float *cval, const uint32_t *skip, cudaStream_t stream)
{
    if (variant < kMpFirst || variant > kMpLast) variant = kMpFirst;
    const int64_t tiles = cdiv(n + nnz, merge_path_items(variant));
    const int kb = mp_shape(variant).carve_kb;
    const int hot = (int)(mp_shape(variant).hot < n ? mp_shape(variant).hot : n);   // within x
#define BOBA_MP(V, MB, MI, C, H)                                                               \
    case V:                                                                                    \
        launch_mp<MB, MI, C, H>(kb, hot, row_ptr, col, val, x, y, n, nnz, part, crow, cval,    \
                                skip, tiles, stream);                                          \
        break;
    switch (variant) {
        BOBA_MP(5, 256, 8, 0, false)
        BOBA_MP(6, 256, 12, 0, false)
        BOBA_MP(7, 512, 8, 0, false)
        BOBA_MP(8, 128, 16, 0, false)
        BOBA_MP(9, 256, 8, 1, false)
        BOBA_MP(10, 256, 8, 2, false)
        BOBA_MP(11, 256, 12, 1, false)
        BOBA_MP(12, 512, 8, 1, false)
        BOBA_MP(13, 256, 16, 1, false)
        BOBA_MP(14, 256, 12, 3, true)
    }
#undef BOBA_MP
    BOBA_TIMED("spmv.fixup", stream,
               k_mp_fixup<<<(unsigned)cdiv(tiles, 256), 256, 0, stream>>>(crow, cval, tiles, n, y,
                                                                           skip));
}

}  // namespace boba

using namespace boba;

extern "C" size_t boba_spmv_workspace_bytes(int64_t n_rows, int64_t nnz)
{
    SpmvLayout L;
    if (!spmv_layout(n_rows, nnz, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_spmv_csr(const int64_t *row_ptr, const int32_t *col,
                                       const float *val, const float *x, float *y, int64_t n_rows,
                                       int64_t nnz, void *ws, size_t ws_bytes, void *stream_)
{
    if (n_rows < 0 || nnz < 0) return BOBA_ERR_INVALID_ARG;
    if (n_rows > kMaxSize || nnz > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n_rows == 0) return BOBA_OK;
    if (row_ptr == nullptr || y == nullptr || x == nullptr) return BOBA_ERR_INVALID_ARG;
    if (nnz > 0 && (col == nullptr || val == nullptr)) return BOBA_ERR_INVALID_ARG;
    if (x == y) return BOBA_ERR_INVALID_ARG;
    SpmvLayout L;
    spmv_layout(n_rows, nnz, L);
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(b + L.count);
    uint32_t *list = reinterpret_cast<uint32_t *>(b + L.list);
    uint32_t *cstart = reinterpret_cast<uint32_t *>(b + L.cstart);
    float *partial = reinterpret_cast<float *>(b + L.partial);
    const uint32_t cap = (uint32_t)L.cap;

    const int tv = tuned_variant(kTuneSpmv, nnz);
    // 0 auto, 1..4: LPR 4, 8, 16, 32; 5..14: merge path, shapes in kMpShapes
    if (tv >= kMpFirst && tv <= kMpLast) {
        int2 *part = reinterpret_cast<int2 *>(b + L.mp_part);
        int32_t *crow = reinterpret_cast<int32_t *>(b + L.mp_crow);
        float *cval = reinterpret_cast<float *>(b + L.mp_cval);
        merge_path_partition(row_ptr, n_rows, nnz, merge_path_items(tv), part, stream);
        merge_path_multiply(tv, row_ptr, col, val, x, y, n_rows, nnz, part, crow, cval, nullptr,
                            stream);
        BOBA_LAUNCH_CHECK();
        return BOBA_OK;
    }
    BOBA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), stream));
    const double avg = (double)nnz / (double)n_rows;
    if (tv == 1) launch_rows<4>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (tv == 2) launch_rows<8>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (tv == 3) launch_rows<16>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (tv == 4) launch_rows<32>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (avg <= 6.0) launch_rows<4>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (avg <= 12.0) launch_rows<8>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else if (avg <= 24.0) launch_rows<16>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    else launch_rows<32>(row_ptr, col, val, x, y, n_rows, cnt, list, cap, dev->status, stream);
    if (nnz > kLongRow) {
        BOBA_TIMED("spmv.long", stream,
                   k_spmv_plan<<<1, 256, 0, stream>>>(row_ptr, cnt, list, cap, cstart));
        const int g = persistent_grid((const void *)k_spmv_chunks, kChunkBlock,
                                      cdiv(nnz, kChunk) + 1);
        BOBA_TIMED("spmv.long", stream,
                   k_spmv_chunks<<<g, kChunkBlock, 0, stream>>>(row_ptr, col, val, x, cnt, list, cap,
                                                                cstart, partial));
        BOBA_TIMED("spmv.long", stream,
                   k_spmv_gather<<<8, 256, 0, stream>>>(cnt, list, cap, cstart, partial, y));
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
