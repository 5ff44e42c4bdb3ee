// boba_reorder_static: the BOBA reorder for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a reorder:
// code running inside a memory-pool or arena that owns all device memory of
// the process, a plug-in hosted by a framework that forbids allocation on its
// hot path, or a real-time loop where an allocation's implicit device
// synchronisation is not acceptable.  They pass their inputs and outputs; the
// scratch this reorder needs lives in a fixed array in the library's own
// device image, which every GPU that loads the library holds until the process
// exits.  No cudaMalloc, cudaFree or allocating library routine is called.
//
// Kernels are the same as boba_reorder_ex's; only the scratch and the launch
// set-up differ.
#include <mutex>

#include "common.cuh"
#include "host.hpp"
#include "reorder_kernels.cuh"

namespace boba {
namespace {

constexpr int64_t kStaticMaxM = 1ll << 22;            // edges
constexpr int64_t kStaticMaxN = 1ll << 20;            // vertices
constexpr size_t kStaticScratchBytes = 10u << 20;     // 10 MiB, holds the layout at the maxima

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: only the address obtained from cudaGetSymbolAddress is passed to
// kernels.  The last word is the status word used when the caller gives none.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes + 256];

constexpr int kMaxDevices = 64;
struct StaticSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;       // device address of g_static_scratch
    int sms = 0;
    int occ_init = 1, occ_first_v = 1, occ_first_s = 1, occ_mark = 1, occ_relabel_v = 1,
        occ_relabel_s = 1;
};
StaticSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

int occ_of(const void *k, int block)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, block, 0) != cudaSuccess || b < 1) {
        (void)cudaGetLastError();
        b = 1;
    }
    return b;
}

// Once per device, with that device current.
boba_status_t setup_for_current_device(const StaticSetup **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOBA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return BOBA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    StaticSetup &s = g_setup[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return BOBA_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return BOBA_ERR_CUDA;
        }
        s.scratch = static_cast<unsigned char *>(p);
        s.occ_init = occ_of((const void *)k_init, 256);
        s.occ_first_v = occ_of((const void *)k_first<true>, kFirstBlock);
        s.occ_first_s = occ_of((const void *)k_first<false>, kFirstBlock);
        s.occ_mark = occ_of((const void *)k_mark, 256);
        s.occ_relabel_v = occ_of((const void *)k_relabel<true>, kRelabelBlock);
        s.occ_relabel_s = occ_of((const void *)k_relabel<false>, kRelabelBlock);
        s.ready = true;
    }
    *out = &s;
    return BOBA_OK;
}

int grid(int sms, int occ, int64_t want)
{
    int64_t g = (int64_t)sms * occ;
    if (want < g) g = want;
    return g < 1 ? 1 : (int)g;
}

}  // namespace
}  // namespace boba

using namespace boba;

// Declared in include/boba.h.
extern "C" boba_status_t boba_reorder_static(const int32_t *src, const int32_t *dst, int64_t m,
                                             int64_t n, int32_t *perm_out, int32_t *src_out,
                                             int32_t *dst_out, uint32_t *error_bits,
                                             void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kStaticMaxM || n > kStaticMaxN) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (perm_out == nullptr) return BOBA_ERR_INVALID_ARG;
    // with no edges there is nothing to read or rewrite: those four may be NULL
    if (m > 0 && (src == nullptr || dst == nullptr || src_out == nullptr || dst_out == nullptr))
        return BOBA_ERR_INVALID_ARG;
    ReorderLayout L;
    if (!reorder_layout(m, n, L) || L.total > kStaticScratchBytes) return BOBA_ERR_TOO_LARGE;

    const StaticSetup *S = nullptr;
    boba_status_t st = setup_for_current_device(&S);
    if (st != BOBA_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    unsigned char *base = S->scratch;

    uint32_t *key = reinterpret_cast<uint32_t *>(base + L.key);
    int32_t *label = reinterpret_cast<int32_t *>(base + L.label);
    uint32_t *grp = reinterpret_cast<uint32_t *>(base + L.grp);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(base + L.bitmap);
    uint64_t *tstat_scan = reinterpret_cast<uint64_t *>(base + L.tstat_scan);
    uint64_t *tstat_emit = reinterpret_cast<uint64_t *>(base + L.tstat_emit);
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + L.counters);
    uint32_t *status = error_bits ? error_bits
                                  : reinterpret_cast<uint32_t *>(base + kStaticScratchBytes);
    const int64_t nzero = (int64_t)((L.zero_end - L.zero_begin) / 4);
    const uint32_t nn = (uint32_t)n;

    // k_init clears everything that must start at zero (bitmap, look-back
    // state, tickets) and sets every key to the sentinel, so no state of an
    // earlier call survives into this one.
    k_init<<<grid(S->sms, S->occ_init, cdiv((L.n4 > nzero ? L.n4 : nzero) / 4, 256)), 256, 0,
             stream>>>(key, L.n4, bitmap, nzero);
    if (m > 0) {
        const bool vec = aligned16(src) && aligned16(dst);
        const int64_t work = cdiv(2 * m, 4 * kFirstBlock * kFirstUnroll);
        if (vec)
            k_first<true><<<grid(S->sms, S->occ_first_v, work), kFirstBlock, 0, stream>>>(
                src, dst, m, nn, key, status);
        else
            k_first<false><<<grid(S->sms, S->occ_first_s, work * 4), kFirstBlock, 0, stream>>>(
                src, dst, m, nn, key, status);
        k_mark<<<grid(S->sms, S->occ_mark, cdiv(L.n4 / 4, 256)), 256, 0, stream>>>(key, L.n4,
                                                                                 bitmap);
        k_scan<<<(unsigned)L.scan_tiles, kScanBlock, 0, stream>>>(bitmap, grp, tstat_scan,
                                                                 counters, L.scan_tiles, status);
    }
    k_emit<<<(unsigned)L.emit_tiles, kEmitBlock, 0, stream>>>(key, nn, bitmap, grp, label,
                                                             perm_out, tstat_emit, counters,
                                                             true, status);
    if (m > 0) {
        const bool vec = aligned16(src) && aligned16(dst) && aligned16(src_out) &&
                         aligned16(dst_out);
        const int64_t work = cdiv(2 * m, 4 * kRelabelBlock * kRelabelUnroll);
        if (vec)
            k_relabel<true><<<grid(S->sms, S->occ_relabel_v, work), kRelabelBlock, 0, stream>>>(
                src, dst, m, nn, label, src_out, dst_out, status);
        else
            k_relabel<false><<<grid(S->sms, S->occ_relabel_s, work * 4), kRelabelBlock, 0,
                               stream>>>(src, dst, m, nn, label, src_out, dst_out, status);
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
