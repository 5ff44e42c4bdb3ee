// COO -> CSR for the pull SpMV of Alg. 3 (arXiv 2306.10410, Sec. 1.2.2):
// rows are destinations, columns are sources, entries of a row keep the input
// edge order, and the entry of edge u -> v holds fp32(1 / outdeg(u)).
//
// A stable LSD radix sort of (key = dst, value = src) with 8-bit digits:
//   k_hist_tiles    per-digit histograms of all passes in one read of dst
//                   (a tile per warp, warp-private shared histograms); for
//                   the reduce-then-scan passes also pass 0's tile counts
//   k_csr_digits    exclusive scan of each pass's 256 digit counts
//   k_csr_pass      one pass: stable in-tile ranking (eight bit-ballots, one
//                   warp match, or per-warp shared-memory OR masks of the
//                   lanes holding each digit, + per-warp digit counters,
//                   items striped so processing order is input order),
//                   per-digit decoupled look-back across tiles, and a
//                   scatter staged through shared memory so that runs of
//                   equal digits are written contiguously (Adinets and
//                   Merrill, "Onesweep", 2022, for the single-pass scheme);
//                   the first pass also counts outdeg(u) over the sources it
//                   carries
//   k_tile_counts,  the reduce-then-scan alternative to the look-back (tuner
//   k_tile_chunk_sums, variants): per-tile digit counts, then a column scan
//   k_tile_apply    of them that gives each tile its digit runs' starts
//   k_csr_ends      ends[k] = one past the last sorted entry of row k, and
//                   val = fp32(1 / outdeg(col)); with two or more passes the
//                   last pass does this itself as it writes its output
//   k_csr_rowptr    row_ptr[v+1] = max over u <= v of ends[u] (a single-pass
//                   max-scan with decoupled look-back), row_ptr[0] = 0
#include <atomic>

#include "common.cuh"
#include "host.hpp"

namespace boba {
namespace {

constexpr int kPassBlock = 512;
constexpr int kPassItems = 8;                        // per thread
// The NBR sorts and boba_sort_by_dst use the pass shape the CSR tuner picks on
// R-MAT 24: ballot ranking with registers capped for three blocks per SM.
constexpr int kPassTile = kPassBlock * kPassItems;  // 4096 items
constexpr int kMaxPasses = 4;                        // 32-bit keys
// How a warp finds the lanes that share its digit: one match instruction,
// eight bit-ballots intersected, or each lane ORs its bit into a per-warp
// shared-memory mask of its digit and reads the mask back.
constexpr int kRankMatch = 0, kRankBallot = 1, kRankOr = 2;
constexpr int kNumCtr = 16;
constexpr int kCountWarps = 8;                   // histogram kernels: 256 threads, a tile per warp

// Look-back status of (tile, digit) for pass p, one u64: the top 4 bits hold
// 2p+1 (aggregate) or 2p+2 (inclusive prefix); anything else (0, or an earlier
// pass's flags) is "not ready".  One array serves all passes of a call.
__device__ __forceinline__ uint64_t pass_flag(int p, bool inclusive)
{
    return (uint64_t)(2 * p + (inclusive ? 2 : 1)) << 60;
}
constexpr uint64_t kPassValMask = (1ull << 60) - 1;

constexpr int kRowRows = 4;                          // rows of 4 vertices per thread
constexpr int kRowTile = 256 * 4 * kRowRows;         // vertices per row_ptr scan tile
constexpr int kCtrRowTicket = 8;

struct CsrLayout {
    int passes;
    int64_t tiles, row_tiles;
    size_t kA, vA, kB, vB, outdeg, hist, dstart, status, counters, ends, rstat, total, zero_begin,
        zero_end;
};

bool csr_layout(int64_t m, int64_t n, CsrLayout &L)
{
    if (m < 0 || n < 0 || m > kMaxSize || n > kMaxSize) return false;
    int bits = 1;
    while (bits < 31 && (1ll << bits) < n) bits++;
    L.passes = (bits + 7) / 8;
    L.tiles = cdiv(m > 0 ? m : 1, kPassTile);
    L.row_tiles = cdiv(n > 0 ? n : 1, kRowTile);
    const size_t mm = (size_t)(m > 0 ? m : 1);
    Carve c;
    L.kA = c.take(mm * 4);
    L.vA = c.take(mm * 4);
    L.kB = c.take(mm * 4);
    L.vB = c.take(mm * 4);
    L.zero_begin = c.off;
    L.outdeg = c.take((size_t)(n > 0 ? n : 1) * 4);
    L.hist = c.take(kMaxPasses * 256 * 4);
    L.status = c.take((size_t)L.tiles * 256 * 8);
    L.counters = c.take(kNumCtr * 4);
    L.ends = c.take((size_t)L.row_tiles * kRowTile * 4);
    L.rstat = c.take((size_t)L.row_tiles * 8);
    L.zero_end = c.off;
    L.dstart = c.take(kMaxPasses * 256 * 4);
    L.total = c.off;
    return true;
}

__global__ void __launch_bounds__(256) k_zero(uint4 *p, int64_t n16)
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z;
}

// Digit histograms of every pass (8-bit digits from bit base_shift on) over
// a key array, one warp per tile of TILE keys with warp-private shared
// histograms, so warps never contend.  With tile_counts it also writes each
// tile's counts of the first digit, which the reduce-then-scan first pass then
// takes instead of its own count kernel.  Keys >= n (n > 0) are reported.
template <int TILE>
__global__ void __launch_bounds__(kCountWarps * 32) k_hist_tiles(
    const uint32_t *__restrict__ keys, int64_t m, int digits, int base_shift, uint32_t n,
    uint32_t *hist, uint32_t *__restrict__ tile_counts, uint32_t *status)
{
    __shared__ uint32_t s_run[kCountWarps][kMaxPasses * 256];   // per warp, all digits
    __shared__ uint32_t s_tile[kCountWarps][256];               // per warp, one tile's first digit
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kCountWarps * kMaxPasses * 256; i += blockDim.x)
        (&s_run[0][0])[i] = 0;
    __syncthreads();
    uint32_t *run = s_run[warp], *th = s_tile[warp];
    uint32_t *first = tile_counts != nullptr ? th : run;
    const int64_t tiles = (m + TILE - 1) / TILE;
    bool bad = false;
    for (int64_t t = (int64_t)blockIdx.x * kCountWarps + warp; t < tiles;
         t += (int64_t)gridDim.x * kCountWarps) {
        if (tile_counts != nullptr) {
#pragma unroll
            for (int i = lane; i < 256; i += 32) th[i] = 0;
            __syncwarp();
        }
        const int64_t t0 = t * TILE;
        const int valid_n = (m - t0) < TILE ? (int)(m - t0) : TILE;
        const uint32_t *k = keys + t0;
        for (int base = 0; base < valid_n; base += 32 * 8) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = base + u * 32 + lane;
                v[u] = j < valid_n ? k[j] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (base + u * 32 + lane < valid_n) {
                    const uint32_t key = v[u];
                    atomicAdd(&first[(key >> base_shift) & 255u], 1u);
                    for (int d = 1; d < digits; ++d)
                        atomicAdd(&run[d * 256 + ((key >> (base_shift + 8 * d)) & 255u)], 1u);
                    bad |= n != 0 && key >= n;
                }
            }
        }
        __syncwarp();
        if (tile_counts != nullptr) {
#pragma unroll
            for (int i = lane; i < 256; i += 32) {
                const uint32_t c = th[i];
                tile_counts[t * 256 + i] = c;
                run[i] += c;
            }
            __syncwarp();
        }
    }
    if (bad) raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
    __syncthreads();
    for (int i = threadIdx.x; i < digits * 256; i += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kCountWarps; ++w) c += s_run[w][i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Launch of k_hist_tiles over the whole key array.
void launch_hist(const char *name, const uint32_t *keys, int64_t m, int digits, int base_shift,
                 uint32_t n, uint32_t *hist, uint32_t *tile_counts, uint32_t *status,
                 cudaStream_t stream)
{
    const int g = persistent_grid((const void *)k_hist_tiles<kPassTile>, kCountWarps * 32,
                                  cdiv(cdiv(m > 0 ? m : 1, kPassTile), kCountWarps));
    BOBA_TIMED(name, stream,
               k_hist_tiles<kPassTile><<<g, kCountWarps * 32, 0, stream>>>(
                   keys, m, digits, base_shift, n, hist, tile_counts, status));
}

// dstart[p][d] = exclusive prefix of hist[p][.] (one block of 256 threads).
__global__ void __launch_bounds__(256) k_csr_digits(const uint32_t *__restrict__ hist,
                                                    uint32_t *__restrict__ dstart, int passes)
{
    __shared__ typename BlockScan<256>::Smem sm;
    for (int p = 0; p < passes; ++p) {
        uint32_t tot;
        const uint32_t ex = BlockScan<256>::exclusive(hist[p * 256 + threadIdx.x], &tot, sm);
        dstart[p * 256 + threadIdx.x] = ex;
        __syncthreads();
    }
}

// One stable LSD pass over digit p (bits 8p .. 8p+7).  BLOCK threads hold
// ITEMS items each; the first 256 threads also own one digit each for the
// cross-tile look-back.  With PRESCAN the global start of each of the tile's
// digit runs is read from tile_base[tile][d] (k_tile_counts, k_tile_chunk_sums
// and k_tile_apply computed it before the pass) instead of the look-back.
template <int BLOCK, int ITEMS, int RANK = kRankMatch, int MINB = 2, bool PRESCAN = false>
__global__ void __launch_bounds__(BLOCK, MINB) k_csr_pass(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t m, int p, const uint32_t *__restrict__ dstart,
    uint64_t *status_lb, uint32_t *counters, uint32_t *status, int digit, int base_shift,
    uint32_t *outdeg = nullptr, uint32_t n = 0, const uint32_t *outdeg_in = nullptr,
    float *val_out = nullptr, uint32_t *ends = nullptr, const uint32_t *tile_base = nullptr)
{
    constexpr int TILE = BLOCK * ITEMS;
    constexpr int WARPS = BLOCK / 32;
    constexpr int WARP_ITEMS = 32 * ITEMS;
    static_assert(BLOCK >= 256, "one thread per digit");
    // the staged tile (TILE keys, then TILE values) in dynamic shared memory
    extern __shared__ __align__(16) uint32_t s_stage[];
    uint32_t *const s_keys = s_stage;
    uint32_t *const s_vals = s_stage + TILE;
    __shared__ uint16_t s_wcnt[WARPS][256];      // per-warp digit counts, then warp prefixes
    __shared__ uint32_t s_tpre[256];              // tile-local exclusive digit offsets
    // global start of this tile's run of digit d minus its tile-local start:
    // sorted tile slot j of digit d goes to s_off[d] + j (mod 2^32)
    __shared__ uint32_t s_off[256];
    constexpr int NBIN = RANK == kRankOr ? 257 : 1;   // digits and the invalid tail
    __shared__ uint32_t s_bins[RANK == kRankOr ? WARPS : 1][NBIN];
    __shared__ typename BlockScan<BLOCK>::Smem sm;
    __shared__ uint32_t s_tile;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (!PRESCAN)
        if (threadIdx.x == 0) s_tile = atomicAdd(&counters[p], 1u);
    for (int i = threadIdx.x; i < WARPS * 256; i += BLOCK) (&s_wcnt[0][0])[i] = 0;
    if constexpr (RANK == kRankOr)
        for (int i = threadIdx.x; i < WARPS * NBIN; i += BLOCK) (&s_bins[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = PRESCAN ? (int64_t)blockIdx.x : (int64_t)s_tile;
    const int64_t t0 = tile * TILE;
    const int shift = base_shift + 8 * digit;
    // items of this tile; tile-local indices and global positions fit 32 bits
    // (m < 2^31)
    const int valid_n = (m - t0) < TILE ? (int)(m - t0) : TILE;
    // every tile but the last is full; the reduce-then-scan shapes rank a
    // full tile without the valid/invalid split (in the look-back shapes it
    // costs registers and measured nothing)
    const bool full = PRESCAN && valid_n == TILE;
    const uint32_t *kin_t = kin + t0, *vin_t = vin + t0;

    // load: item (warp, k, lane) is tile index warp*WARP_ITEMS + k*32 + lane, so
    // the k-major / lane-minor processing order of a warp is the input order
    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int j = warp * WARP_ITEMS + k * 32 + lane;
        if (j < valid_n) {
            key[k] = __ldcs(kin_t + j);
            val[k] = __ldcs(vin_t + j);
        } else {
            key[k] = 0xFFFFFFFFu;
            val[k] = 0;
        }
    }
    if (outdeg != nullptr) {
        // the first pass of the CSR build also counts outdeg(u) over the
        // values (the sources): fire-and-forget L2 reductions beside the ranking
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            if (warp * WARP_ITEMS + k * 32 + lane < valid_n) {
                if (val[k] < n) atomicAdd(&outdeg[val[k]], 1u);
                else raise_status(status, BOBA_ERR_ID_OUT_OF_RANGE);
            }
        }
    }
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const bool valid = full || warp * WARP_ITEMS + k * 32 + lane < valid_n;
        const uint32_t d = valid ? ((key[k] >> shift) & 255u) : 256u;
        unsigned peers;
        if constexpr (RANK == kRankOr) {
            atomicOr(&s_bins[warp][d], 1u << lane);
            __syncwarp();
            peers = s_bins[warp][d];
        } else if constexpr (RANK == kRankBallot) {
            // lanes with the same digit: intersect 8 bit-ballots (and the
            // valid/invalid split) instead of one match instruction
            if (full) {
                peers = kFull;
            } else {
                const unsigned vm = __ballot_sync(kFull, valid);
                peers = valid ? vm : ~vm;
            }
            // per bit: the lanes whose bit b matches this lane's, that is
            // the ballot of the bit, inverted where this lane's bit is clear.
            // In PTX the one predicate drives both the vote and the
            // inversion; the C++ select between bm and ~bm issued more ALU
            // instructions in this ALU-bound loop (radix pass on 2^28 keys:
            // 1.93 ms, now 1.82-1.85 ms)
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                asm("{\n\t.reg .pred p;\n\t.reg .b32 m;\n\t"
                    "setp.ne.u32 p, %1, 0;\n\t"
                    "vote.sync.ballot.b32 m, p, 0xffffffff;\n\t"
                    "@!p not.b32 m, m;\n\t"
                    "and.b32 %0, %0, m;\n\t}"
                    : "+r"(peers) : "r"(d & (1u << b)));
            }
        } else {
            peers = __match_any_sync(kFull, d);
        }
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = s_wcnt[warp][d];
            s_wcnt[warp][d] = (uint16_t)(old + __popc(peers));
        }
        old = __shfl_sync(kFull, old, leader);
        rank[k] = old + __popc(peers & lt);
        __syncwarp();
        if constexpr (RANK == kRankOr) {
            // every lane has read its mask: the group's first lane clears it
            // for the next round
            if (lane == leader) s_bins[warp][d] = 0;
            __syncwarp();
        }
    }
    __syncthreads();
    // digit d = threadIdx.x (< 256): tile count, warp prefixes, tile-local offsets
    const int d = threadIdx.x;
    uint32_t cnt = 0;
    if (d < 256) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = (uint16_t)cnt;
            cnt += c;
        }
    }
    uint32_t tot;
    const uint32_t tpre = BlockScan<BLOCK>::exclusive(cnt, &tot, sm);
    if (d < 256 && PRESCAN) {
        s_tpre[d] = tpre;
        s_off[d] = tile_base[tile * 256 + d] - tpre;
    } else if (d < 256) {
        s_tpre[d] = tpre;
        // per-digit look-back across tiles, reading 8 predecessors per round trip
        uint64_t *st = status_lb + tile * 256 + d;
        if (tile == 0) {
            st_relaxed_u64(st, pass_flag(p, true) | cnt);
            s_off[d] = dstart[digit * 256 + d] - tpre;
        } else {
            st_relaxed_u64(st, pass_flag(p, false) | cnt);
            const uint64_t fa = pass_flag(p, false), fp = pass_flag(p, true);
            uint64_t excl = 0;
            int64_t t = tile - 1;
            uint64_t tstart = 0;
            uint32_t spins = 0;
            while (t >= 0) {
                uint64_t w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    w[j] = (t - j >= 0) ? ld_relaxed_u64(status_lb + (t - j) * 256 + d) : fp;
                int used = 0;
                bool done = false;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (done || used != j) continue;
                    const uint64_t f = w[j] & ~kPassValMask;
                    if (f == fp) { excl += w[j] & kPassValMask; done = true; }
                    else if (f == fa) { excl += w[j] & kPassValMask; ++used; }
                }
                if (done) break;
                t -= used;
                if (used == 0) {
                    if ((++spins & 255u) == 1u || spins >= kMaxSpins) {
                        const uint64_t now = globaltimer_ns();
                        if (tstart == 0) tstart = now;
                        if (now - tstart > kTimeoutNs || spins >= kMaxSpins) {
                            raise_status(status, BOBA_ERR_TIMEOUT);
                            break;
                        }
                    }
                    __nanosleep(32);
                }
            }
            st_relaxed_u64(st, fp | ((excl + cnt) & kPassValMask));
            s_off[d] = dstart[digit * 256 + d] + (uint32_t)excl - tpre;
        }
    }
    __syncthreads();
    // stage the tile in shared memory in sorted order
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (warp * WARP_ITEMS + k * 32 + lane < valid_n) {
            const uint32_t dd = (key[k] >> shift) & 255u;
            const uint32_t pos = s_tpre[dd] + s_wcnt[warp][dd] + rank[k];
            s_keys[pos] = key[k];
            s_vals[pos] = val[k];
        }
    }
    __syncthreads();
    // write out: consecutive threads write consecutive slots of a digit run
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int j = k * BLOCK + threadIdx.x;
        if (j < valid_n) {
            const uint32_t kk = s_keys[j];
            const uint32_t vv = s_vals[j];
            const uint32_t dd = (kk >> shift) & 255u;
            const uint32_t g = s_off[dd] + (uint32_t)j;
            __stcs(vout + g, vv);
            if (ends == nullptr) {
                __stcs(kout + g, kk);
                continue;
            }
            // the last pass of the CSR build: the sorted keys are not kept;
            // instead val = fp32(1 / outdeg(col)) and the row ends.  Inside
            // the tile's run of digit dd the keys are sorted, so a key whose
            // successor in the run differs ends here; a key at the end of the
            // run may continue in a later tile, so it offers its end by max.
            const uint32_t dg = vv < n ? __ldg(outdeg_in + vv) : 0u;
            float r;
            if (dg == 0) r = 0.0f;
            else if (dg < (1u << 24)) r = __frcp_rn((float)dg);      // exact operand, IEEE rounding
            else r = (float)(1.0 / (double)dg);
            __stcs(val_out + g, r);
            if (kk < n) {
                const int run_end = dd < 255u ? (int)s_tpre[dd + 1] : (int)valid_n;
                if (j + 1 < run_end) {
                    if (s_keys[j + 1] != kk) ends[kk] = g + 1;
                } else {
                    atomicMax(&ends[kk], g + 1);
                }
            }
        }
    }
}

// Reduce-then-scan alternative to the look-back (the PRESCAN passes).
constexpr int kChunkTiles = 256;                 // tiles per block of the count scan
constexpr int kCtrPrescan = 12;                  // counters slot: ticket of the chunk-sum blocks

// counts[t][d] = items of tile t (TILE items, the pass's tiles) whose digit is
// d.  One warp counts a whole tile into a warp-private shared histogram, so
// nothing but __syncwarp orders it; the grid strides over the tiles.
template <int TILE>
__global__ void __launch_bounds__(kCountWarps * 32) k_tile_counts(
    const uint32_t *__restrict__ kin, int64_t m, int shift, int64_t tiles,
    uint32_t *__restrict__ counts)
{
    __shared__ uint32_t s_h[kCountWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *h = s_h[warp];
    for (int64_t t = (int64_t)blockIdx.x * kCountWarps + warp; t < tiles;
         t += (int64_t)gridDim.x * kCountWarps) {
#pragma unroll
        for (int i = lane; i < 256; i += 32) h[i] = 0;
        __syncwarp();
        const int64_t t0 = t * TILE;
        const int valid_n = (m - t0) < TILE ? (int)(m - t0) : TILE;
        const uint32_t *k = kin + t0;
        for (int base = 0; base < valid_n; base += 32 * 8) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = base + u * 32 + lane;
                v[u] = j < valid_n ? k[j] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (base + u * 32 + lane < valid_n) atomicAdd(&h[(v[u] >> shift) & 255u], 1u);
        }
        __syncwarp();
#pragma unroll
        for (int i = lane; i < 256; i += 32) counts[t * 256 + i] = h[i];
        __syncwarp();
    }
}

// csum[c][d] = sum of counts[t][d] over the kChunkTiles tiles of chunk c; the
// last block to finish (by ticket) then rewrites csum[c][d] as dstart[d] plus
// the sum over the chunks before c: where chunk c's run of digit d starts.
// The ticket starts at 0 (the workspace is cleared) and the last block puts it
// back to 0 for the next pass.
__global__ void __launch_bounds__(256) k_tile_chunk_sums(const uint32_t *__restrict__ counts,
                                                         int64_t tiles, int64_t chunks,
                                                         uint32_t *csum,
                                                         const uint32_t *__restrict__ dstart_p,
                                                         uint32_t *ticket)
{
    __shared__ bool s_last;
    const int d = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int64_t t1 = (c + 1) * kChunkTiles < tiles ? (c + 1) * kChunkTiles : tiles;
    uint32_t s = 0;
#pragma unroll 16
    for (int64_t t = c * kChunkTiles; t < t1; ++t) s += counts[t * 256 + d];
    csum[c * 256 + d] = s;
    __threadfence();
    __syncthreads();
    if (d == 0) s_last = atomicAdd(ticket, 1u) == (uint32_t)chunks - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (d == 0) *ticket = 0;
    uint32_t base = dstart_p[d];
    for (int64_t q = 0; q < chunks; q += 16) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = q + u < chunks ? __ldcg(&csum[(q + u) * 256 + d]) : 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (q + u < chunks) csum[(q + u) * 256 + d] = base;
            base += v[u];
        }
    }
}

// counts[t][d] <- where tile t's run of digit d starts: its chunk's start plus
// the counts of the chunk's earlier tiles.
__global__ void __launch_bounds__(256) k_tile_apply(uint32_t *counts, int64_t tiles,
                                                    const uint32_t *__restrict__ cbase)
{
    const int d = threadIdx.x;
    const int64_t c = blockIdx.x;
    uint32_t base = cbase[c * 256 + d];
    const int64_t t_begin = c * kChunkTiles;
    const int64_t t1 = t_begin + kChunkTiles < tiles ? t_begin + kChunkTiles : tiles;
    constexpr int G = 16;                         // rows loaded before they are rewritten
    for (int64_t t = t_begin; t < t1; t += G) {
        uint32_t v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) v[g] = t + g < t1 ? counts[(t + g) * 256 + d] : 0u;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (t + g < t1) counts[(t + g) * 256 + d] = base;
            base += v[g];
        }
    }
}

// One radix pass of the CSR build in a given shape (the tuner's variants).
// Every shape's tile holds at least kPassTile items, so the look-back status
// array sized for kPassTile tiles serves all of them.
struct CsrPassArgs {
    const uint32_t *kin, *vin;
    uint32_t *kout, *vout;
    int64_t m;
    int p;
    const uint32_t *dstart;
    uint64_t *lb;
    uint32_t *ctr, *status, *outdeg;
    uint32_t n;
    const uint32_t *outdeg_in;
    float *val_out;
    uint32_t *ends;
    int digit = 0, base_shift = 0;   // key bits base_shift + 8 digit .. + 7; 0, 0: digit p
    bool counts_ready = false;       // the tile counts are in place (k_hist_tiles wrote them)
};

template <int BLOCK, int ITEMS, int RANK, int MINB, bool PRESCAN = false>
void csr_pass_launch(const char *name, const CsrPassArgs &a, cudaStream_t stream)
{
    constexpr int TILE = BLOCK * ITEMS;
    static_assert(TILE >= kPassTile, "the status array is sized for kPassTile tiles");
    constexpr size_t smem = (size_t)TILE * 8;
    // static plus dynamic shared memory above 48 KB needs the opt-in, and
    // several shapes are there (the OR masks alone take 16 KB): set it for
    // every shape, once per device
    static std::atomic<uint64_t> done{0};          // devices whose attribute is set
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if ((done.load() & bit) == 0) {
        cudaFuncSetAttribute((const void *)k_csr_pass<BLOCK, ITEMS, RANK, MINB, PRESCAN>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        done.fetch_or(bit);
    }
    const unsigned tiles = (unsigned)cdiv(a.m > 0 ? a.m : 1, TILE);
    uint32_t *tile_base = nullptr;
    if constexpr (PRESCAN) {
        // the look-back status array (8 bytes per tile and digit of kPassTile
        // tiles) holds the counts (4 bytes per tile and digit) and the chunk sums
        tile_base = reinterpret_cast<uint32_t *>(a.lb);
        uint32_t *csum = tile_base + (size_t)tiles * 256;
        const unsigned chunks = (unsigned)cdiv(tiles, kChunkTiles);
        uint32_t *ticket = a.ctr + kCtrPrescan;
        const int gc = persistent_grid((const void *)k_tile_counts<TILE>, kCountWarps * 32,
                                       cdiv(tiles, kCountWarps));
        static_assert(TILE == kPassTile, "k_hist_tiles writes the first pass's counts per kPassTile");
        if (!a.counts_ready)
            BOBA_TIMED("csr.prescan", stream,
                       k_tile_counts<TILE><<<gc, kCountWarps * 32, 0, stream>>>(
                           a.kin, a.m, a.base_shift + 8 * a.digit, tiles, tile_base));
        BOBA_TIMED("csr.prescan", stream,
                   k_tile_chunk_sums<<<chunks, 256, 0, stream>>>(
                       tile_base, tiles, chunks, csum, a.dstart + a.digit * 256, ticket));
        BOBA_TIMED("csr.prescan", stream,
                   k_tile_apply<<<chunks, 256, 0, stream>>>(tile_base, tiles, csum));
    }
    BOBA_TIMED(name, stream,
               k_csr_pass<BLOCK, ITEMS, RANK, MINB, PRESCAN><<<tiles, BLOCK, smem, stream>>>(
                   a.kin, a.vin, a.kout, a.vout, a.m, a.p, a.dstart, a.lb, a.ctr, a.status,
                   a.digit, a.base_shift, a.outdeg, a.n, a.outdeg_in, a.val_out, a.ends,
                   tile_base));
}

// The pass the NBR sorts and boba_sort_by_dst use: the default shape, with
// the reduce-then-scan offsets from 2^22 keys on (measured faster there; the
// three extra launches per pass cost more than they save below).
constexpr int64_t kPrescanMin = 1ll << 22;

void sort_pass(const char *name, const CsrPassArgs &a, cudaStream_t stream)
{
    if (a.m >= kPrescanMin)
        csr_pass_launch<kPassBlock, kPassItems, kRankBallot, 3, true>(name, a, stream);
    else
        csr_pass_launch<kPassBlock, kPassItems, kRankBallot, 3>(name, a, stream);
}

// ends[k] = 1 + index of the last sorted entry with key k (0 if none);
// val[i] = fp32(1 / outdeg(col[i])), correctly rounded.
__global__ void __launch_bounds__(256) k_csr_ends(const uint32_t *__restrict__ skeys,
                                                  const int32_t *__restrict__ col, int64_t m,
                                                  uint32_t n, const uint32_t *__restrict__ outdeg,
                                                  uint32_t *__restrict__ ends,
                                                  float *__restrict__ val)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint32_t k = skeys[i];
        if (k < n && (i == m - 1 || skeys[i + 1] != k)) ends[k] = (uint32_t)(i + 1);
        const uint32_t c = (uint32_t)__ldcs(col + i);
        const uint32_t dg = c < n ? __ldg(outdeg + c) : 0u;
        float r;
        if (dg == 0) r = 0.0f;
        else if (dg < (1u << 24)) r = __frcp_rn((float)dg);      // exact operand, IEEE rounding
        else r = (float)(1.0 / (double)dg);
        __stcs(val + i, r);
    }
}

// row_ptr[0] = 0, row_ptr[v+1] = max over u <= v of ends[u]: an inclusive
// max-scan, single pass with decoupled look-back over vertex tiles.
__global__ void __launch_bounds__(256) k_csr_rowptr(const uint32_t *__restrict__ ends, int64_t n,
                                                    int64_t *__restrict__ row_ptr, uint64_t *tstat,
                                                    uint32_t *counters, uint32_t *status)
{
    __shared__ typename BlockScan<256, OpMax32>::Smem sm;
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(&counters[kCtrRowTicket], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    // row q of the tile: vertices tile*T + q*1024 .., thread t's four at 4t
    __shared__ uint32_t s_rowmax[kRowRows];
    uint32_t run[kRowRows][4], within[kRowRows];
#pragma unroll
    for (int q = 0; q < kRowRows; ++q) {
        const int64_t vq = tile * kRowTile + q * 1024 + 4 * (int64_t)threadIdx.x;
        const uint4 e = *reinterpret_cast<const uint4 *>(ends + vq);   // padded, zero beyond n
        run[q][0] = e.x;
        run[q][1] = max(run[q][0], e.y);
        run[q][2] = max(run[q][1], e.z);
        run[q][3] = max(run[q][2], e.w);
        uint32_t rt;
        within[q] = BlockScan<256, OpMax32>::exclusive(run[q][3], &rt, sm);
        if (threadIdx.x == 0) s_rowmax[q] = rt;
        __syncthreads();                   // the scan's shared words are reused
    }
    uint32_t row_before[kRowRows], tot = 0;
#pragma unroll
    for (int q = 0; q < kRowRows; ++q) {
        row_before[q] = max(tot, within[q]);
        tot = max(tot, s_rowmax[q]);
    }
    if (threadIdx.x < 32) {
        const uint64_t p = lookback_exclusive<OpMax>(tstat, tile, tot, status);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    if (tile == 0 && threadIdx.x == 0) row_ptr[0] = 0;
#pragma unroll
    for (int q = 0; q < kRowRows; ++q) {
        const int64_t vq = tile * kRowTile + q * 1024 + 4 * (int64_t)threadIdx.x;
        const uint32_t pre = max((uint32_t)s_prefix, row_before[q]);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (vq + j < n) row_ptr[vq + j + 1] = (int64_t)max(pre, run[q][j]);
    }
}

__global__ void k_rowptr_zero(int64_t *row_ptr, int64_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x)
        row_ptr[v] = 0;
}

// ---------------------------------------------------------------------------
// NBR locality metric (Sec. 5.2): for each row with a non-empty neighbour
// set N(v), lines(N(v)) / |N(v)| with N(v) the distinct column IDs of the row
// and lines the distinct ids_per_line-wide blocks of IDs they fall in; NBR is
// the mean over those rows.  The columns of every row are sorted by two
// stable radix sorts (by column, then by row), after which distinct values
// and distinct lines are counted by comparing neighbours.
// ---------------------------------------------------------------------------

// rows[p] = r for every entry p of row r (a warp per row).
__global__ void __launch_bounds__(256) k_expand_rows(const int64_t *__restrict__ row_ptr,
                                                     int64_t n_rows, uint32_t *__restrict__ rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n_rows; r += nw) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        for (int64_t p = b + lane; p < e; p += 32) rows[p] = (uint32_t)r;
    }
}

// Per block: sum of lines/distinct over its rows (fixed order) and the count
// of non-empty rows.  A warp per row; rows go to warps round-robin.
__global__ void __launch_bounds__(256) k_nbr_rows(const int64_t *__restrict__ row_ptr,
                                                  const uint32_t *__restrict__ scol, int64_t n_rows,
                                                  uint32_t line, double *__restrict__ bsum,
                                                  unsigned long long *__restrict__ bcnt)
{
    __shared__ double s_sum[8];
    __shared__ unsigned long long s_cnt[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * 8 + warp;
    const int64_t nw = (int64_t)gridDim.x * 8;
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (int64_t r = w; r < n_rows; r += nw) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        if (e == b) continue;
        uint32_t distinct = 0, lines = 0;
        for (int64_t p = b + lane; p < e; p += 32) {
            const uint32_t c = scol[p];
            const bool first = p == b;
            const uint32_t pc = first ? 0u : scol[p - 1];
            distinct += (first || c != pc) ? 1u : 0u;
            lines += (first || c / line != pc / line) ? 1u : 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            distinct += __shfl_xor_sync(kFull, distinct, o);
            lines += __shfl_xor_sync(kFull, lines, o);
        }
        sum += (double)lines / (double)distinct;          // same value in every lane
        ++cnt;
    }
    if (lane == 0) { s_sum[warp] = sum; s_cnt[warp] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int i = 0; i < 8; ++i) { t += s_sum[i]; c += s_cnt[i]; }
        bsum[blockIdx.x] = t;
        bcnt[blockIdx.x] = c;
    }
}

__global__ void k_nbr_final(const double *bsum, const unsigned long long *bcnt, int blocks,
                            double *out_sum, unsigned long long *out_cnt)
{
    double t = 0.0;
    unsigned long long c = 0;
    for (int i = 0; i < blocks; ++i) { t += bsum[i]; c += bcnt[i]; }
    *out_sum = t;
    *out_cnt = c;
}

constexpr int kNbrBlocks = 1216;       // fixed, so the reduction order never changes

struct NbrLayout {
    int passes;
    int64_t tiles;
    size_t rows, kA, vA, kB, vB, hist1, hist2, status, counters, zero_begin, zero_end, dst1, dst2,
        bsum, bcnt, out, total;
};

bool nbr_layout(int64_t n_rows, int64_t nnz, NbrLayout &L)
{
    if (n_rows < 0 || nnz < 0 || n_rows > kMaxSize || nnz > kMaxSize) return false;
    int bits = 1;
    while (bits < 31 && (1ll << bits) < n_rows) bits++;
    L.passes = (bits + 7) / 8;
    L.tiles = cdiv(nnz > 0 ? nnz : 1, kPassTile);
    const size_t mm = (size_t)(nnz > 0 ? nnz : 1) * 4;
    Carve c;
    L.rows = c.take(mm);
    L.kA = c.take(mm);
    L.vA = c.take(mm);
    L.kB = c.take(mm);
    L.vB = c.take(mm);
    L.zero_begin = c.off;
    L.hist1 = c.take(kMaxPasses * 256 * 4);
    L.hist2 = c.take(kMaxPasses * 256 * 4);
    L.status = c.take((size_t)L.tiles * 256 * 8);
    L.counters = c.take(kNumCtr * 4);
    L.zero_end = c.off;
    L.dst1 = c.take(kMaxPasses * 256 * 4);
    L.dst2 = c.take(kMaxPasses * 256 * 4);
    L.bsum = c.take(kNbrBlocks * 8);
    L.bcnt = c.take(kNbrBlocks * 8);
    L.out = c.take(16);
    L.total = c.off;
    return true;
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" size_t boba_nbr_workspace_bytes(int64_t n_rows, int64_t nnz)
{
    NbrLayout L;
    if (!nbr_layout(n_rows, nnz, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_nbr(const int64_t *row_ptr, const int32_t *col, int64_t n_rows,
                                  int64_t nnz, int64_t ids_per_line, double *nbr_out,
                                  int64_t *rows_counted, void *ws, size_t ws_bytes, void *stream_)
{
    if (n_rows < 0 || nnz < 0 || ids_per_line < 1 || ids_per_line > 0x7FFFFFFF)
        return BOBA_ERR_INVALID_ARG;
    if (n_rows > kMaxSize || nnz > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (nbr_out == nullptr) return BOBA_ERR_INVALID_ARG;
    if (n_rows == 0 || nnz == 0) {
        *nbr_out = 0.0;
        if (rows_counted) *rows_counted = 0;
        return BOBA_OK;
    }
    if (row_ptr == nullptr || col == nullptr) return BOBA_ERR_INVALID_ARG;
    NbrLayout L;
    nbr_layout(n_rows, nnz, L);
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    auto U = [&](size_t off) { return reinterpret_cast<uint32_t *>(b + off); };
    uint64_t *lb = reinterpret_cast<uint64_t *>(b + L.status);
    const int64_t zero16 = (int64_t)(L.zero_end - L.zero_begin) / 16;
    const int gz = persistent_grid((const void *)k_zero, 256, cdiv(zero16, 256));
    BOBA_TIMED("nbr", stream, k_zero<<<gz, 256, 0, stream>>>(reinterpret_cast<uint4 *>(b + L.zero_begin), zero16));
    const int gr = persistent_grid((const void *)k_expand_rows, 256, cdiv(n_rows * 32, 256));
    BOBA_TIMED("nbr", stream, k_expand_rows<<<gr, 256, 0, stream>>>(row_ptr, n_rows, U(L.rows)));
    // the first sort's pass 0 reads col in this order, so its tile counts come
    // with the histogram; the second sort's input order is the first's output
    const bool pre = nnz >= kPrescanMin;
    launch_hist("nbr", reinterpret_cast<const uint32_t *>(col), nnz, L.passes, 0, 0u, U(L.hist1),
                pre ? reinterpret_cast<uint32_t *>(lb) : nullptr, dev->status, stream);
    launch_hist("nbr", U(L.rows), nnz, L.passes, 0, 0u, U(L.hist2), nullptr, dev->status, stream);
    BOBA_TIMED("nbr", stream, k_csr_digits<<<1, 256, 0, stream>>>(U(L.hist1), U(L.dst1), L.passes));
    BOBA_TIMED("nbr", stream, k_csr_digits<<<1, 256, 0, stream>>>(U(L.hist2), U(L.dst2), L.passes));
    // sort 1: by column (values: rows)
    const uint32_t *kin = reinterpret_cast<const uint32_t *>(col), *vin = U(L.rows);
    for (int p = 0; p < L.passes; ++p) {
        uint32_t *ko = (p & 1) ? U(L.kB) : U(L.kA), *vo = (p & 1) ? U(L.vB) : U(L.vA);
        sort_pass(
            "nbr", CsrPassArgs{kin, vin, ko, vo, nnz, p, U(L.dst1), lb, U(L.counters), dev->status,
                               nullptr, 0, nullptr, nullptr, nullptr, p, 0, p == 0},
            stream);
        kin = ko;
        vin = vo;
    }
    // sort 2: by row (values: columns), stable, so columns stay sorted in a row
    BOBA_TIMED("nbr", stream, k_zero<<<gz, 256, 0, stream>>>(reinterpret_cast<uint4 *>(b + L.status),
                                                             (int64_t)(L.zero_end - L.status) / 16));
    // inputs of sort 2: rows (the values of sort 1) as keys, columns as values;
    // outputs alternate between two free buffers and the two input buffers
    uint32_t *rbuf = const_cast<uint32_t *>(vin), *cbuf = const_cast<uint32_t *>(kin);
    uint32_t *fb[2];
    int nf = 0;
    for (uint32_t *q : {U(L.rows), U(L.kA), U(L.vA), U(L.kB), U(L.vB)})
        if (q != rbuf && q != cbuf && nf < 2) fb[nf++] = q;
    kin = rbuf;
    vin = cbuf;
    for (int p = 0; p < L.passes; ++p) {
        uint32_t *ko = (p & 1) ? rbuf : fb[0], *vo = (p & 1) ? cbuf : fb[1];
        sort_pass(
            "nbr", CsrPassArgs{kin, vin, ko, vo, nnz, p, U(L.dst2), lb, U(L.counters), dev->status,
                               nullptr, 0, nullptr, nullptr, nullptr, p, 0},
            stream);
        kin = ko;
        vin = vo;
    }
    double *bsum = reinterpret_cast<double *>(b + L.bsum);
    unsigned long long *bcnt = reinterpret_cast<unsigned long long *>(b + L.bcnt);
    BOBA_TIMED("nbr", stream,
               k_nbr_rows<<<kNbrBlocks, 256, 0, stream>>>(row_ptr, vin, n_rows,
                                                          (uint32_t)ids_per_line, bsum, bcnt));
    double *dsum = reinterpret_cast<double *>(b + L.out);
    unsigned long long *dcnt = reinterpret_cast<unsigned long long *>(b + L.out + 8);
    BOBA_TIMED("nbr", stream, k_nbr_final<<<1, 1, 0, stream>>>(bsum, bcnt, kNbrBlocks, dsum, dcnt));
    double hs = 0.0;
    unsigned long long hc = 0;
    BOBA_CUDA_TRY(cudaMemcpyAsync(&hs, dsum, 8, cudaMemcpyDeviceToHost, stream));
    BOBA_CUDA_TRY(cudaMemcpyAsync(&hc, dcnt, 8, cudaMemcpyDeviceToHost, stream));
    BOBA_CUDA_TRY(cudaStreamSynchronize(stream));
    *nbr_out = hc ? hs / (double)hc : 0.0;
    if (rows_counted) *rows_counted = (int64_t)hc;
    return BOBA_OK;
}

// ---------------------------------------------------------------------------
// Stable sort (or binning) of a COO by destination, the remedy Sec. 5.6
// suggests for edge lists in random order before running BOBA.
// ---------------------------------------------------------------------------

namespace boba {
namespace {

struct SortLayout {
    int passes, bits;
    int64_t tiles;
    size_t kA, vA, kB, vB, zero_begin, hist, status, counters, zero_end, dstart, total;
};

bool sort_layout(int64_t m, int64_t n, SortLayout &L)
{
    if (m < 0 || n < 0 || m > kMaxSize || n > kMaxSize) return false;
    int bits = 1;
    while (bits < 31 && (1ll << bits) < n) bits++;
    L.bits = bits;
    L.passes = (bits + 7) / 8;
    L.tiles = cdiv(m > 0 ? m : 1, kPassTile);
    const size_t mm = (size_t)(m > 0 ? m : 1) * 4;
    Carve c;
    L.kA = c.take(mm);
    L.vA = c.take(mm);
    L.kB = c.take(mm);
    L.vB = c.take(mm);
    L.zero_begin = c.off;
    L.hist = c.take(kMaxPasses * 256 * 4);
    L.status = c.take((size_t)L.tiles * 256 * 8);
    L.counters = c.take(kNumCtr * 4);
    L.zero_end = c.off;
    L.dstart = c.take(kMaxPasses * 256 * 4);
    L.total = c.off;
    return true;
}

}  // namespace
}  // namespace boba

extern "C" size_t boba_sort_by_dst_workspace_bytes(int64_t m, int64_t n)
{
    SortLayout L;
    if (!sort_layout(m, n, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_sort_by_dst(const int32_t *src, const int32_t *dst, int64_t m,
                                          int64_t n, int32_t *src_out, int32_t *dst_out,
                                          int top_digit_only, void *ws, size_t ws_bytes,
                                          void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (m == 0) return BOBA_OK;
    if (!src || !dst || !src_out || !dst_out) return BOBA_ERR_INVALID_ARG;
    SortLayout L;
    sort_layout(m, n, L);
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    char *b = static_cast<char *>(ws);
    auto U = [&](size_t off) { return reinterpret_cast<uint32_t *>(b + off); };
    const int64_t zero16 = (int64_t)(L.zero_end - L.zero_begin) / 16;
    const int gz = persistent_grid((const void *)k_zero, 256, cdiv(zero16, 256));
    BOBA_TIMED("sort", stream, k_zero<<<gz, 256, 0, stream>>>(reinterpret_cast<uint4 *>(b + L.zero_begin), zero16));
    // full sort: digits 0 .. passes-1 from bit 0; binning: one digit, the top 8
    // significant bits of a ceil(log2 n)-bit ID
    const int digits = top_digit_only ? 1 : L.passes;
    const int base = top_digit_only ? (L.bits > 8 ? L.bits - 8 : 0) : 0;
    launch_hist("sort", reinterpret_cast<const uint32_t *>(dst), m, digits, base, 0u, U(L.hist),
                m >= kPrescanMin ? U(L.status) : nullptr, dev->status, stream);
    BOBA_TIMED("sort", stream, k_csr_digits<<<1, 256, 0, stream>>>(U(L.hist), U(L.dstart), digits));
    const uint32_t *kin = reinterpret_cast<const uint32_t *>(dst);
    const uint32_t *vin = reinterpret_cast<const uint32_t *>(src);
    for (int d = 0, p = 0; d < digits; ++d, ++p) {
        const bool last = d == digits - 1;
        uint32_t *ko = last ? reinterpret_cast<uint32_t *>(dst_out) : ((p & 1) ? U(L.kB) : U(L.kA));
        uint32_t *vo = last ? reinterpret_cast<uint32_t *>(src_out) : ((p & 1) ? U(L.vB) : U(L.vA));
        sort_pass(
            "sort", CsrPassArgs{kin, vin, ko, vo, m, p, U(L.dstart),
                                reinterpret_cast<uint64_t *>(b + L.status), U(L.counters),
                                dev->status, nullptr, 0, nullptr, nullptr, nullptr, d, base,
                                d == 0},
            stream);
        kin = ko;
        vin = vo;
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

extern "C" size_t boba_coo_to_csr_workspace_bytes(int64_t m, int64_t n)
{
    CsrLayout L;
    if (!csr_layout(m, n, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_coo_to_csr(const int32_t *src, const int32_t *dst, int64_t m,
                                         int64_t n, int64_t *row_ptr, int32_t *col_out,
                                         float *val_out, void *ws, size_t ws_bytes, void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if (row_ptr == nullptr) return BOBA_ERR_INVALID_ARG;
    if (m > 0 && (src == nullptr || dst == nullptr || col_out == nullptr || val_out == nullptr))
        return BOBA_ERR_INVALID_ARG;
    CsrLayout L;
    csr_layout(m, n, L);
    if (ws == nullptr || ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (m == 0) {
        BOBA_TIMED("csr.finish", stream,
                   k_rowptr_zero<<<(unsigned)cdiv(n + 1, 256) < 1024 ? (unsigned)cdiv(n + 1, 256) : 1024u,
                                   256, 0, stream>>>(row_ptr, n));
        BOBA_LAUNCH_CHECK();
        return BOBA_OK;
    }
    char *b = static_cast<char *>(ws);
    uint32_t *kA = reinterpret_cast<uint32_t *>(b + L.kA), *vA = reinterpret_cast<uint32_t *>(b + L.vA);
    uint32_t *kB = reinterpret_cast<uint32_t *>(b + L.kB), *vB = reinterpret_cast<uint32_t *>(b + L.vB);
    uint32_t *outdeg = reinterpret_cast<uint32_t *>(b + L.outdeg);
    uint32_t *ends = reinterpret_cast<uint32_t *>(b + L.ends);
    uint32_t *hist = reinterpret_cast<uint32_t *>(b + L.hist);
    uint32_t *dstart = reinterpret_cast<uint32_t *>(b + L.dstart);
    uint64_t *lb = reinterpret_cast<uint64_t *>(b + L.status);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(b + L.counters);
    const uint32_t nn = (uint32_t)n;

    {
        const int64_t n16 = (int64_t)(L.zero_end - L.zero_begin) / 16;
        const int g = persistent_grid((const void *)k_zero, 256, cdiv(n16, 256));
        BOBA_TIMED("csr.zero", stream,
                   k_zero<<<g, 256, 0, stream>>>(reinterpret_cast<uint4 *>(b + L.zero_begin), n16));
    }
    // variant 0 (untuned): the look-back passes, or from kPrescanMin keys on
    // their reduce-then-scan form (variant 8), measured faster there
    int tv = tuned_variant(kTuneCsr, m);
    if (tv == 0 && m >= kPrescanMin) tv = 8;
    const bool prescan = tv == 8 || tv == 9;        // the reduce-then-scan shapes (tiles of kPassTile)
    launch_hist("csr.hist", reinterpret_cast<const uint32_t *>(dst), m, L.passes, 0, nn, hist,
                prescan ? reinterpret_cast<uint32_t *>(lb) : nullptr, dev->status, stream);
    BOBA_TIMED("csr.digits", stream,
               k_csr_digits<<<1, 256, 0, stream>>>(hist, dstart, L.passes));
    const uint32_t *kin = reinterpret_cast<const uint32_t *>(dst);
    const uint32_t *vin = reinterpret_cast<const uint32_t *>(src);
    for (int p = 0; p < L.passes; ++p) {
        const bool last = p == L.passes - 1;
        uint32_t *ko = (p & 1) ? kB : kA;
        uint32_t *vo = last ? reinterpret_cast<uint32_t *>(col_out) : ((p & 1) ? vB : vA);
        // pass 0 counts outdeg; with two or more passes the last one also
        // writes val and the row ends (outdeg is complete by then)
        uint32_t *od = p == 0 ? outdeg : nullptr;
        const bool fuse = last && L.passes > 1;
        uint32_t *ends_p = fuse ? ends : nullptr;
        float *val_p = fuse ? val_out : nullptr;
        const uint32_t *od_in = fuse ? outdeg : nullptr;
        const CsrPassArgs pa{kin, vin, ko, vo, m, p, dstart, lb, ctr, dev->status, od, nn,
                             od_in, val_p, ends_p, p, 0, prescan && p == 0};
        switch (tv) {
        case 1: csr_pass_launch<512, 8, kRankBallot, 2>("csr.pass", pa, stream); break;
        case 2: csr_pass_launch<512, 8, kRankMatch, 2>("csr.pass", pa, stream); break;
        case 3: csr_pass_launch<512, 8, kRankOr, 3>("csr.pass", pa, stream); break;
        case 4: csr_pass_launch<256, 16, kRankBallot, 3>("csr.pass", pa, stream); break;
        case 5: csr_pass_launch<256, 16, kRankOr, 3>("csr.pass", pa, stream); break;
        case 6: csr_pass_launch<384, 16, kRankBallot, 2>("csr.pass", pa, stream); break;
        case 7: csr_pass_launch<512, 16, kRankBallot, 1>("csr.pass", pa, stream); break;
        case 8: csr_pass_launch<512, 8, kRankBallot, 3, true>("csr.pass", pa, stream); break;
        case 9: csr_pass_launch<256, 16, kRankOr, 3, true>("csr.pass", pa, stream); break;
        default: csr_pass_launch<512, 8, kRankBallot, 3>("csr.pass", pa, stream); break;
        }
        kin = ko;
        vin = vo;
    }
    {
        if (L.passes == 1) {
            const int g = persistent_grid((const void *)k_csr_ends, 256, cdiv(m, 256));
            BOBA_TIMED("csr.finish", stream,
                       k_csr_ends<<<g, 256, 0, stream>>>(kin, col_out, m, nn, outdeg, ends,
                                                         val_out));
        }
        BOBA_TIMED("csr.finish", stream,
                   k_csr_rowptr<<<(unsigned)L.row_tiles, 256, 0, stream>>>(
                       ends, n, row_ptr, reinterpret_cast<uint64_t *>(b + L.rstat), ctr,
                       dev->status));
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
