// Host-side helpers shared by the translation units of libboba.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/boba.h"

namespace boba {

constexpr int64_t kMaxSize = 2147483647ll;   // 2^31 - 1

struct DeviceInfo {
    int device = -1;
    int sms = 0;
    uint32_t *status = nullptr;   // per-device status word (cudaMalloc'd once)
};

// Info for the current device; lazily created.  Returns nullptr on CUDA error.
const DeviceInfo *device_info();

// Blocks per SM for `kernel` at `block` threads (cached by kernel pointer).
int occupancy(const void *kernel, int block, size_t dyn_smem = 0);

// A persistent grid: SMs x resident blocks, capped by `max_blocks` (>= 1).
int persistent_grid(const void *kernel, int block, int64_t max_blocks, size_t dyn_smem = 0);

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// Workspace carving helper: successive 256-byte-aligned regions.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

// Kernel timing: when enabled, launches made through BOBA_TIMED are bracketed
// by CUDA events on their stream and accumulated per kernel name.
bool timing_on();
void timing_begin(const char *name, cudaStream_t s, int *slot);
void timing_end(int slot, cudaStream_t s);

// Autotuned choices: the variant index picked for a kernel family and a size
// (bucketed by log2 of the size), or 0 (the default variant) if none.
enum TuneKernel { kTuneFirst = 0, kTuneRelabel = 1, kTuneBatched = 2, kTuneSpmv = 3,
                  kTuneCsr = 4, kTuneKernels = 5 };
int tuned_variant(int kernel, int64_t size);
int size_class(int64_t size);

// Merge-path SpMV (spmv.cu), shared with the iterative callers.  `variant` is a
// tuned SpMV variant 5..13 (anything else means 5): it fixes the block shape,
// the path items per tile and the shared-memory carve-out.  The partition depends on row_ptr only, so an
// iterative caller computes it once.  A non-null `skip` pointing at a nonzero
// word makes the multiply's kernels return at once.
int merge_path_items(int variant);
void merge_path_partition(const int64_t *row_ptr, int64_t n, int64_t nnz, int items, int2 *part,
                          cudaStream_t stream);
void merge_path_multiply(int variant, const int64_t *row_ptr, const int32_t *col, const float *val,
                         const float *x, float *y, int64_t n, int64_t nnz, const int2 *part,
                         int32_t *crow, float *cval, const uint32_t *skip, cudaStream_t stream);

}  // namespace boba

// BOBA_TIMED("name", stream, kernel<<<g, b, smem, stream>>>(args));
// Every launch also sits in an NVTX range of the same name (header-only NVTX 3;
// a no-op unless a profiler is attached), so a profiler can filter by phase.
#define BOBA_TIMED(name, stream, ...)                                  \
    do {                                                               \
        int _slot = -1;                                                \
        nvtxRangePushA(name);                                          \
        if (::boba::timing_on()) ::boba::timing_begin(name, stream, &_slot); \
        __VA_ARGS__;                                                   \
        if (_slot >= 0) ::boba::timing_end(_slot, stream);             \
        nvtxRangePop();                                                \
    } while (0)

#define BOBA_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            (void)cudaGetLastError();                         \
            return BOBA_ERR_CUDA;                             \
        }                                                     \
    } while (0)

#define BOBA_LAUNCH_CHECK()                                   \
    do {                                                      \
        cudaError_t _e = cudaGetLastError();                  \
        if (_e != cudaSuccess) return BOBA_ERR_CUDA;          \
    } while (0)
