// boba_reorder_host: the reorder of a graph held in host memory, with the
// copies overlapped with the kernels.
//
// The edge list moves to the device in chunks on an internal copy stream;
// the first-occurrence pass runs on each chunk as soon as it has arrived
// (keys of a chunk use global positions, so chunks combine by AtomicMin in
// any order).  After the labels are known, each chunk is relabelled and its
// result copied back on a second internal stream while the next chunk is
// relabelled.  The caller's stream is ordered before and after the call as if
// all the work ran on it.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "host.hpp"
#include "reorder_kernels.cuh"

namespace boba {

// The position-based first-occurrence kernel and the relabel kernel (reorder.cu).
template <bool VEC>
__global__ void k_first_at(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           int64_t m, uint32_t n, uint32_t *key, uint32_t *status, int64_t pos_src,
                           int64_t pos_dst);

namespace {

constexpr int64_t kChunk = 1ll << 24;       // edges per chunk (64 MiB per endpoint array)

struct HostIo {
    bool ready = false;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> events;
    std::mutex mu;                          // calls on one device enqueue one at a time
};
HostIo g_io[64];
std::mutex g_io_init;

HostIo *host_io()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_io_init);
    HostIo &h = g_io[dev];
    if (!h.ready) {
        if (cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h.d2h, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        h.ready = true;
    }
    return &h;
}

cudaEvent_t event_at(HostIo &h, size_t i)
{
    while (h.events.size() <= i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        h.events.push_back(e);
    }
    return h.events[i];
}

struct HostLayout {
    size_t src, dst, so, dout, perm, rws, total;
    ReorderLayout R;
};

bool host_layout(int64_t m, int64_t n, HostLayout &L)
{
    if (!reorder_layout(m, n, L.R)) return false;
    const size_t mm = (size_t)(m > 0 ? m : 1) * 4;
    Carve c;
    L.src = c.take(mm);
    L.dst = c.take(mm);
    L.so = c.take(mm);
    L.dout = c.take(mm);
    L.perm = c.take((size_t)(n > 0 ? n : 1) * 4);
    L.rws = c.take(L.R.total);
    L.total = c.off;
    return true;
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" size_t boba_reorder_host_workspace_bytes(int64_t m, int64_t n)
{
    HostLayout L;
    if (m < 0 || n < 0 || m > kMaxSize || n > kMaxSize || !host_layout(m, n, L)) return 0;
    return L.total;
}

extern "C" boba_status_t boba_reorder_host(const int32_t *src_h, const int32_t *dst_h, int64_t m,
                                           int64_t n, int32_t *perm_h, int32_t *src_out_h,
                                           int32_t *dst_out_h, void *ws, size_t ws_bytes,
                                           void *stream_)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (perm_h == nullptr || ws == nullptr) return BOBA_ERR_INVALID_ARG;
    if (m > 0 && (!src_h || !dst_h || !src_out_h || !dst_out_h)) return BOBA_ERR_INVALID_ARG;
    HostLayout L;
    host_layout(m, n, L);
    if (ws_bytes < L.total || !aligned256(ws)) return BOBA_ERR_WORKSPACE;
    const DeviceInfo *dev = device_info();
    HostIo *io = host_io();
    if (!dev || !io) return BOBA_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    std::lock_guard<std::mutex> lk(io->mu);
    char *b = static_cast<char *>(ws);
    int32_t *src = reinterpret_cast<int32_t *>(b + L.src), *dst = reinterpret_cast<int32_t *>(b + L.dst);
    int32_t *so = reinterpret_cast<int32_t *>(b + L.so), *dout = reinterpret_cast<int32_t *>(b + L.dout);
    int32_t *perm = reinterpret_cast<int32_t *>(b + L.perm);
    char *rb = b + L.rws;
    const ReorderLayout &R = L.R;

    ReorderArgs a;
    a.src = src;
    a.dst = dst;
    a.m = m;
    a.n = (uint32_t)n;
    a.key = reinterpret_cast<uint32_t *>(rb + R.key);
    a.label = reinterpret_cast<int32_t *>(rb + R.label);
    a.perm = perm;
    a.bitmap = reinterpret_cast<uint32_t *>(rb + R.bitmap);
    a.grp = reinterpret_cast<uint32_t *>(rb + R.grp);
    a.tstat_scan = reinterpret_cast<uint64_t *>(rb + R.tstat_scan);
    a.tstat_emit = reinterpret_cast<uint64_t *>(rb + R.tstat_emit);
    a.counters = reinterpret_cast<uint32_t *>(rb + R.counters);
    a.nwords = R.nwords;
    a.scan_tiles = R.scan_tiles;
    a.emit_tiles = R.emit_tiles;
    a.status = dev->status;
    a.src_out = so;
    a.dst_out = dout;
    a.label_vec = true;

    size_t ev = 0;
    auto next_event = [&]() { return event_at(*io, ev++); };
    const int64_t chunks = cdiv(m, kChunk);

    // the copy streams start after everything already queued on the caller's stream
    cudaEvent_t e_start = next_event();
    if (!e_start) return BOBA_ERR_CUDA;
    BOBA_CUDA_TRY(cudaEventRecord(e_start, s));
    BOBA_CUDA_TRY(cudaStreamWaitEvent(io->h2d, e_start, 0));
    BOBA_CUDA_TRY(cudaStreamWaitEvent(io->d2h, e_start, 0));
    {
        const int64_t nzero = (int64_t)((R.zero_end - R.zero_begin) / 4);
        const int64_t work = cdiv((R.n4 > nzero ? R.n4 : nzero) / 4, 256);
        const int g = persistent_grid((const void *)k_init, 256, work);
        BOBA_TIMED("reorder.init", s, k_init<<<g, 256, 0, s>>>(a.key, R.n4, a.bitmap, nzero));
    }
    // 1. copies in, first occurrence per chunk as it lands
    for (int64_t c = 0; c < chunks; ++c) {
        const int64_t e0 = c * kChunk, len = (m - e0) < kChunk ? (m - e0) : kChunk;
        BOBA_CUDA_TRY(cudaMemcpyAsync(src + e0, src_h + e0, (size_t)len * 4, cudaMemcpyHostToDevice, io->h2d));
        BOBA_CUDA_TRY(cudaMemcpyAsync(dst + e0, dst_h + e0, (size_t)len * 4, cudaMemcpyHostToDevice, io->h2d));
        cudaEvent_t e = next_event();
        if (!e) return BOBA_ERR_CUDA;
        BOBA_CUDA_TRY(cudaEventRecord(e, io->h2d));
        BOBA_CUDA_TRY(cudaStreamWaitEvent(s, e, 0));
        const int64_t work = cdiv(2 * len, 4 * kFirstBlock * kFirstUnroll);
        const int g = persistent_grid((const void *)k_first_at<true>, kFirstBlock, work);
        BOBA_TIMED("reorder.first", s,
                   k_first_at<true><<<g, kFirstBlock, 0, s>>>(src + e0, dst + e0, len, a.n, a.key,
                                                              a.status, e0, m + e0));
    }
    // 2. ranks, labels, perm
    {
        const int gm = persistent_grid((const void *)k_mark, 256, cdiv(R.n4 / 4, 256));
        if (m > 0) {
            BOBA_TIMED("reorder.mark", s, k_mark<<<gm, 256, 0, s>>>(a.key, R.n4, a.bitmap));
            BOBA_TIMED("reorder.scan", s,
                       k_scan<<<(unsigned)a.scan_tiles, kScanBlock, 0, s>>>(
                           a.bitmap, a.grp, a.tstat_scan, a.counters, a.scan_tiles, a.status));
        }
        BOBA_TIMED("reorder.emit", s,
                   k_emit<<<(unsigned)a.emit_tiles, kEmitBlock, 0, s>>>(
                       a.key, a.n, a.bitmap, a.grp, a.label, a.perm, a.tstat_emit, a.counters,
                       a.label_vec, a.status));
        cudaEvent_t e = next_event();
        if (!e) return BOBA_ERR_CUDA;
        BOBA_CUDA_TRY(cudaEventRecord(e, s));
        BOBA_CUDA_TRY(cudaStreamWaitEvent(io->d2h, e, 0));
        BOBA_CUDA_TRY(cudaMemcpyAsync(perm_h, perm, (size_t)n * 4, cudaMemcpyDeviceToHost, io->d2h));
    }
    // 3. relabel per chunk, copies out as each chunk is done
    for (int64_t c = 0; c < chunks; ++c) {
        const int64_t e0 = c * kChunk, len = (m - e0) < kChunk ? (m - e0) : kChunk;
        const int64_t work = cdiv(2 * len, 4 * kRelabelBlock * kRelabelUnroll);
        const int g = persistent_grid((const void *)k_relabel<true>, kRelabelBlock, work);
        BOBA_TIMED("reorder.relabel", s,
                   k_relabel<true><<<g, kRelabelBlock, 0, s>>>(src + e0, dst + e0, len, a.n, a.label,
                                                               so + e0, dout + e0, a.status));
        cudaEvent_t e = next_event();
        if (!e) return BOBA_ERR_CUDA;
        BOBA_CUDA_TRY(cudaEventRecord(e, s));
        BOBA_CUDA_TRY(cudaStreamWaitEvent(io->d2h, e, 0));
        BOBA_CUDA_TRY(cudaMemcpyAsync(src_out_h + e0, so + e0, (size_t)len * 4, cudaMemcpyDeviceToHost, io->d2h));
        BOBA_CUDA_TRY(cudaMemcpyAsync(dst_out_h + e0, dout + e0, (size_t)len * 4, cudaMemcpyDeviceToHost, io->d2h));
    }
    // 4. the caller's stream continues after the last copy out
    cudaEvent_t e_end = next_event();
    if (!e_end) return BOBA_ERR_CUDA;
    BOBA_CUDA_TRY(cudaEventRecord(e_end, io->d2h));
    BOBA_CUDA_TRY(cudaStreamWaitEvent(s, e_end, 0));
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
