// boba_probe_gather: the rate of random 4-byte loads on this GPU, from global
// memory, from a block's shared memory and from the distributed shared memory
// of a thread-block cluster.
//
// This is a measurement aid, not a step of the method.  The first-occurrence
// pass (Alg. 2, Sec. 4.4) and the relabel (Sec. 5.3) each look up one entry
// of an n-sized array per endpoint, at an index that is random for a randomly
// labelled input.  The probe issues the same kind of load with no stream
// beside it, so its rate is the ceiling those two passes can reach with one
// lookup per endpoint, and the rates of the on-chip forms say what keeping
// the array in shared or distributed shared memory would buy.
//
// Indices come from the murmur3 32-bit finaliser (Appleby, MurmurHash3,
// public domain) of a per-thread counter, masked to a power-of-two table.
#include <cooperative_groups.h>

#include "common.cuh"
#include "host.hpp"

namespace cg = cooperative_groups;

namespace boba {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeUnroll = 8;     // independent loads in flight per thread

__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// mode 0: loads through L1TEX from a global table of mask+1 words.
__global__ void __launch_bounds__(kProbeBlock) k_probe_global(const uint32_t *__restrict__ table,
                                                              uint32_t mask, int64_t per_thread,
                                                              uint32_t seed, uint32_t *out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ctr = fmix32(seed ^ (t * 0x9E3779B9u));
    uint32_t acc = 0;
    for (int64_t k = 0; k < per_thread; k += kProbeUnroll) {
        uint32_t v[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) v[u] = __ldg(table + (fmix32(ctr + u) & mask));
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc += v[u];
        ctr += kProbeUnroll;
    }
    out[t] = acc;
}

// mode 1: the block copies mask+1 words of the table into its shared memory,
// then loads from there.
__global__ void __launch_bounds__(kProbeBlock) k_probe_shared(const uint32_t *__restrict__ table,
                                                              uint32_t mask, int64_t per_thread,
                                                              uint32_t seed, uint32_t *out)
{
    extern __shared__ uint32_t s_tab[];
    for (uint32_t i = threadIdx.x; i <= mask; i += blockDim.x) s_tab[i] = table[i];
    __syncthreads();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ctr = fmix32(seed ^ (t * 0x9E3779B9u));
    uint32_t acc = 0;
    for (int64_t k = 0; k < per_thread; k += kProbeUnroll) {
        uint32_t v[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) v[u] = s_tab[fmix32(ctr + u) & mask];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc += v[u];
        ctr += kProbeUnroll;
    }
    out[t] = acc;
}

// mode 2: a cluster of C blocks holds C * (mask+1) words, mask+1 per block;
// every load picks a block of the cluster and a word in it.
__global__ void __launch_bounds__(kProbeBlock) k_probe_cluster(const uint32_t *__restrict__ table,
                                                               uint32_t mask, int64_t per_thread,
                                                               uint32_t seed, uint32_t *out)
{
    extern __shared__ uint32_t s_tab[];
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t nblk = cluster.num_blocks();
    const uint32_t rank = cluster.block_rank();
    for (uint32_t i = threadIdx.x; i <= mask; i += blockDim.x)
        s_tab[i] = table[(size_t)rank * (mask + 1) + i];
    cluster.sync();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ctr = fmix32(seed ^ (t * 0x9E3779B9u));
    uint32_t acc = 0;
    for (int64_t k = 0; k < per_thread; k += kProbeUnroll) {
        uint32_t v[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            const uint32_t h = fmix32(ctr + u);
            const uint32_t *p = cluster.map_shared_rank(s_tab + (h & mask), (h >> 24) % nblk);
            v[u] = *p;
        }
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc += v[u];
        ctr += kProbeUnroll;
    }
    out[t] = acc;
    cluster.sync();          // no block leaves while others may still read its shared memory
}

}  // namespace
}  // namespace boba

using namespace boba;

extern "C" boba_status_t boba_probe_gather(int mode, const uint32_t *table, int64_t table_words,
                                           int64_t loads_per_thread, int cluster, uint32_t *out,
                                           int64_t out_words, int64_t *loads_issued, void *stream_)
{
    if (mode < 0 || mode > 2 || table == nullptr || out == nullptr || loads_issued == nullptr)
        return BOBA_ERR_INVALID_ARG;
    if (table_words < 1 || table_words > (1ll << 31) || (table_words & (table_words - 1)) != 0)
        return BOBA_ERR_INVALID_ARG;
    if (loads_per_thread < kProbeUnroll || loads_per_thread % kProbeUnroll != 0)
        return BOBA_ERR_INVALID_ARG;
    const DeviceInfo *dev = device_info();
    if (!dev) return BOBA_ERR_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    int64_t per_block_words = table_words;
    if (mode == 2) {
        if (cluster < 2 || cluster > 16 || (cluster & (cluster - 1)) != 0 ||
            table_words % cluster != 0)
            return BOBA_ERR_INVALID_ARG;
        per_block_words = table_words / cluster;
    }
    const size_t smem = mode == 0 ? 0 : (size_t)per_block_words * 4;
    if (smem > 227u * 1024u) return BOBA_ERR_INVALID_ARG;
    const uint32_t mask = (uint32_t)(per_block_words - 1);
    const uint32_t seed = 0x2306u;
    const void *kern = mode == 0 ? (const void *)k_probe_global
                       : mode == 1 ? (const void *)k_probe_shared : (const void *)k_probe_cluster;
    if (smem > 48u * 1024u)
        BOBA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    if (mode == 0 || mode == 1) {
        int64_t g = persistent_grid(kern, kProbeBlock, out_words / kProbeBlock, smem);
        if (g < 1) return BOBA_ERR_INVALID_ARG;
        if (mode == 0)
            BOBA_TIMED("probe.gather", stream,
                       k_probe_global<<<(unsigned)g, kProbeBlock, 0, stream>>>(
                           table, mask, loads_per_thread, seed, out));
        else
            BOBA_TIMED("probe.gather", stream,
                       k_probe_shared<<<(unsigned)g, kProbeBlock, smem, stream>>>(
                           table, mask, loads_per_thread, seed, out));
        *loads_issued = g * kProbeBlock * loads_per_thread;
    } else {
        if (cluster > 8)
            BOBA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(kProbeBlock);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        cfg.gridDim = dim3((unsigned)cluster);
        BOBA_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg));
        if (clusters < 1) return BOBA_ERR_INVALID_ARG;
        int64_t g = (int64_t)clusters * cluster;
        while (g > out_words / kProbeBlock && g > cluster) g -= cluster;
        if (g * kProbeBlock > out_words) return BOBA_ERR_INVALID_ARG;
        cfg.gridDim = dim3((unsigned)g);
        cudaError_t e = cudaSuccess;
        BOBA_TIMED("probe.gather", stream,
                   e = cudaLaunchKernelEx(&cfg, k_probe_cluster, table, mask, loads_per_thread,
                                          seed, out));
        BOBA_CUDA_TRY(e);
        *loads_issued = g * kProbeBlock * loads_per_thread;
    }
    BOBA_LAUNCH_CHECK();
    return BOBA_OK;
}
