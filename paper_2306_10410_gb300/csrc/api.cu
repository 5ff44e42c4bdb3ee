// Library-level entry points: device bookkeeping, the status word, the
// cached-workspace form of boba_reorder, and status strings.
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "host.hpp"

namespace boba {

namespace {
std::mutex g_mu;
std::map<int, DeviceInfo> g_dev;
std::map<std::pair<int, const void *>, int> g_occ;

struct CachedWs {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::map<std::pair<int, void *>, CachedWs> g_ws;   // (device, stream) -> workspace
}  // namespace

const DeviceInfo *device_info()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) return &it->second;
    DeviceInfo d;
    d.device = dev;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMalloc(&d.status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(d.status, 0, sizeof(uint32_t)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return &(g_dev[dev] = d);
}

int occupancy(const void *kernel, int block, size_t dyn_smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_occ.find({dev, kernel});
        if (it != g_occ.end()) return it->second;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, block, dyn_smem) !=
            cudaSuccess || blocks < 1) {
        (void)cudaGetLastError();
        blocks = 1;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_occ[{dev, kernel}] = blocks;
    return blocks;
}

int persistent_grid(const void *kernel, int block, int64_t max_blocks, size_t dyn_smem)
{
    const DeviceInfo *d = device_info();
    const int sms = d ? d->sms : 1;
    int64_t g = (int64_t)sms * occupancy(kernel, block, dyn_smem);
    if (max_blocks < g) g = max_blocks;
    if (g < 1) g = 1;
    return (int)g;
}

// Self-test of the bounded wait: tile 1 looks back at tile 0, whose status
// word nothing ever publishes (it stays 0).  The wait must give up after
// timeout_ns, record BOBA_ERR_TIMEOUT and let the kernel finish.
__global__ void k_selftest_lookback(uint64_t *tstat, uint32_t *status, uint64_t timeout_ns,
                                    uint64_t *out)
{
    if (threadIdx.x < 32) {
        const uint64_t p = lookback_exclusive(tstat, 1, 5, status, false, timeout_ns);
        if (threadIdx.x == 0) *out = p;
    }
}

}  // namespace boba

using namespace boba;

extern "C" boba_status_t boba_selftest_wait_timeout(uint64_t timeout_ns, void *scratch,
                                                    void *stream)
{
    if (scratch == nullptr || timeout_ns == 0 || timeout_ns > kTimeoutNs) return BOBA_ERR_INVALID_ARG;
    const DeviceInfo *d = device_info();
    if (!d) return BOBA_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *tstat = static_cast<uint64_t *>(scratch);
    BOBA_CUDA_TRY(cudaMemsetAsync(tstat, 0, 3 * sizeof(uint64_t), s));
    k_selftest_lookback<<<1, 32, 0, s>>>(tstat, d->status, timeout_ns, tstat + 2);
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}

extern "C" boba_status_t boba_reorder(const int32_t *src, const int32_t *dst, int64_t m,
                                      int64_t n, int32_t *perm_out, int32_t *src_out,
                                      int32_t *dst_out, void *stream)
{
    if (m < 0 || n < 0) return BOBA_ERR_INVALID_ARG;
    if (m > kMaxSize || n > kMaxSize) return BOBA_ERR_TOO_LARGE;
    if (n == 0 && m > 0) return BOBA_ERR_INVALID_ARG;
    if (n == 0) return BOBA_OK;
    if (src_out == nullptr || dst_out == nullptr) return BOBA_ERR_INVALID_ARG;
    const size_t need = boba_reorder_workspace_bytes(m, n);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BOBA_ERR_CUDA;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        CachedWs &c = g_ws[{dev, stream}];
        if (c.bytes < need) {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) {
                (void)cudaGetLastError();
                return BOBA_ERR_CUDA;
            }
            if (cap != cudaStreamCaptureStatusNone) return BOBA_ERR_WORKSPACE;
            if (c.ptr) {
                // earlier calls on this stream may still read the old buffer
                if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess ||
                    cudaFree(c.ptr) != cudaSuccess) {
                    (void)cudaGetLastError();
                    return BOBA_ERR_CUDA;
                }
                c.ptr = nullptr;
                c.bytes = 0;
            }
            const size_t grow = need + need / 8;
            if (cudaMalloc(&c.ptr, grow) != cudaSuccess) {
                (void)cudaGetLastError();
                c.ptr = nullptr;
                return BOBA_ERR_WORKSPACE;
            }
            c.bytes = grow;
        }
        ws = c.ptr;
    }
    return boba_reorder_ex(src, dst, m, n, perm_out, src_out, dst_out, nullptr, ws, need, stream);
}

extern "C" boba_status_t boba_stream_status(void *stream)
{
    const DeviceInfo *d = device_info();
    if (!d) return BOBA_ERR_CUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOBA_ERR_CUDA;
    }
    uint32_t bits = 0;
    if (cudaMemcpy(&bits, d->status, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(d->status, 0, sizeof(uint32_t)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return BOBA_ERR_CUDA;
    }
    // most severe first
    static const boba_status_t order[] = {BOBA_ERR_TIMEOUT, BOBA_ERR_INVALID_ARG,
                                          BOBA_ERR_ID_OUT_OF_RANGE, BOBA_ERR_TOO_LARGE,
                                          BOBA_ERR_WORKSPACE, BOBA_ERR_CUDA};
    for (boba_status_t s : order)
        if (bits & (1u << (int)s)) return s;
    return BOBA_OK;
}

extern "C" const char *boba_status_string(boba_status_t s)
{
    switch (s) {
    case BOBA_OK: return "BOBA_OK";
    case BOBA_ERR_INVALID_ARG: return "BOBA_ERR_INVALID_ARG";
    case BOBA_ERR_ID_OUT_OF_RANGE: return "BOBA_ERR_ID_OUT_OF_RANGE";
    case BOBA_ERR_TOO_LARGE: return "BOBA_ERR_TOO_LARGE";
    case BOBA_ERR_WORKSPACE: return "BOBA_ERR_WORKSPACE";
    case BOBA_ERR_TIMEOUT: return "BOBA_ERR_TIMEOUT";
    case BOBA_ERR_CUDA: return "BOBA_ERR_CUDA";
    }
    return "BOBA_ERR_UNKNOWN";
}

extern "C" const char *boba_version(void) { return "boba-gb300 0.1 (sm_103a)"; }
