// Autotuner: for each kernel family with several correct launch variants
// (block size and loads in flight of the first-occurrence and relabel
// streams, their warp-aggregated and bulk-copy forms, the schedule of the
// batched path, the SpMV kernel and shape --
// lanes per row, or merge-path block, items and shared-memory carve-out --
// and the ranking, tile shape and offset scheme (look-back or
// reduce-then-scan) of the radix passes), time every variant on the caller's
// data and keep the fastest for that size class (log2 of the size) on this
// device.  Integer results must equal the default's bit for bit (a variant
// that differs is skipped); the SpMV shapes differ only in the order of fp32
// sums, and one whose product is further than the error bound (relative L2
// 1e-5) from the default's is skipped too.  Choices can be saved to and loaded from
// a text file keyed by GPU name.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "host.hpp"

namespace boba {
namespace {

constexpr int kClasses = 64;
// The fp32 SpMV is within 1e-5 (relative L2) of the fp64 product; a tuned
// variant must also stay within that of the default variant's fp32 result.
constexpr double kSpmvTuneRelL2 = 1e-5;
constexpr int kMaxDev = 64;
constexpr int kVariants[kTuneKernels] = {8, 8, 9, 15, 10};   // first, relabel, batched, spmv, csr
const char *kNames[kTuneKernels] = {"first", "relabel", "batched", "spmv", "csr"};

std::mutex g_tmu;
signed char g_table[kMaxDev][kTuneKernels][kClasses];
bool g_init = false;

void init_table()
{
    if (!g_init) {
        memset(g_table, -1, sizeof(g_table));
        g_init = true;
    }
}

int cur_dev()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return (d >= 0 && d < kMaxDev) ? d : -1;
}

std::string dev_name()
{
    cudaDeviceProp p;
    int d = cur_dev();
    if (d < 0 || cudaGetDeviceProperties(&p, d) != cudaSuccess) {
        (void)cudaGetLastError();
        return "unknown";
    }
    std::string s = p.name;
    for (char &c : s)
        if (c == ' ' || c == '|') c = '_';
    return s;
}

__global__ void k_count_diff(const int32_t *a, const int32_t *b, int64_t n, unsigned long long *cnt)
{
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        local += a[i] != b[i];
    if (local) atomicAdd(cnt, local);
}

// Number of differing 32-bit words between device arrays a and b.
int64_t count_diff(const void *a, const void *b, int64_t words, unsigned long long *dcnt,
                   cudaStream_t s)
{
    if (words <= 0) return 0;
    cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long), s);
    k_count_diff<<<256, 256, 0, s>>>(static_cast<const int32_t *>(a), static_cast<const int32_t *>(b),
                                     words, dcnt);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, dcnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return (int64_t)h;
}

// sums[0] += (a - b)^2, sums[1] += b^2 over n floats, in fp64.
__global__ void k_sq_diff(const float *a, const float *b, int64_t n, double *sums)
{
    double d2 = 0.0, b2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        d2 += d * d;
        b2 += (double)b[i] * (double)b[i];
    }
    if (d2 != 0.0) atomicAdd(&sums[0], d2);
    if (b2 != 0.0) atomicAdd(&sums[1], b2);
}

// Relative L2 distance ||a - b|| / ||b|| of two device float arrays (-1 on a
// CUDA error; ||a|| if b is all zero).
double rel_l2(const float *a, const float *b, int64_t n, double *dsums, cudaStream_t s)
{
    if (n <= 0) return 0.0;
    cudaMemsetAsync(dsums, 0, 2 * sizeof(double), s);
    k_sq_diff<<<256, 256, 0, s>>>(a, b, n, dsums);
    double h[2] = {0.0, 0.0};
    cudaMemcpyAsync(h, dsums, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1.0;
    }
    return h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
}

template <class F>
double time_ms(F &&fn, int reps, cudaStream_t s)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        fn();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t.empty() ? 0.0 : t[t.size() / 2];
}

void set_entry(int kernel, int cls, int v)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    init_table();
    const int d = cur_dev();
    if (d >= 0 && kernel >= 0 && kernel < kTuneKernels && cls >= 0 && cls < kClasses)
        g_table[d][kernel][cls] = (signed char)v;
}

}  // namespace

int size_class(int64_t size)
{
    int c = 0;
    while (c < kClasses - 1 && (1ll << (c + 1)) <= size) ++c;
    return c;
}

int tuned_variant(int kernel, int64_t size)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    init_table();
    const int d = cur_dev();
    if (d < 0 || kernel < 0 || kernel >= kTuneKernels) return 0;
    const int v = g_table[d][kernel][size_class(size)];
    return v < 0 ? 0 : v;
}

}  // namespace boba

using namespace boba;

extern "C" int boba_tune_get(int kernel, int64_t size) { return tuned_variant(kernel, size); }

extern "C" void boba_tune_set(int kernel, int64_t size, int variant)
{
    if (kernel < 0 || kernel >= kTuneKernels) return;
    if (variant < -1 || variant >= kVariants[kernel]) return;
    set_entry(kernel, size_class(size), variant);
}

extern "C" void boba_tune_reset(void)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    memset(g_table, -1, sizeof(g_table));
    g_init = true;
}

extern "C" boba_status_t boba_tune_reorder(const int32_t *src, const int32_t *dst, int64_t m,
                                           int64_t n, int32_t *perm_out, int32_t *src_out,
                                           int32_t *dst_out, void *ws, size_t ws_bytes, int reps,
                                           int *chosen, void *stream_)
{
    if (reps < 1 || m <= 0 || n <= 0 || !perm_out || !src_out || !dst_out) return BOBA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    const int cls = size_class(m);
    void *ref = nullptr;
    unsigned long long *dcnt = nullptr;
    const size_t ref_bytes = (size_t)(2 * m + n) * 4;
    if (cudaMalloc(&ref, ref_bytes) != cudaSuccess || cudaMalloc(&dcnt, 8) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ref) cudaFree(ref);
        return BOBA_ERR_CUDA;
    }
    int32_t *rperm = static_cast<int32_t *>(ref), *rso = rperm + n, *rdo = rso + m;
    auto run = [&] {
        return boba_reorder_ex(src, dst, m, n, perm_out, src_out, dst_out, nullptr, ws, ws_bytes, s);
    };
    boba_status_t st = BOBA_OK;
    set_entry(kTuneFirst, cls, 0);
    set_entry(kTuneRelabel, cls, 0);
    if ((st = run()) != BOBA_OK) goto done;
    cudaMemcpyAsync(rperm, perm_out, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(rso, src_out, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(rdo, dst_out, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < 2 && st == BOBA_OK; ++k) {
        const int kernel = k == 0 ? kTuneFirst : kTuneRelabel;
        int best = 0;
        double best_ms = 1e30;
        for (int v = 0; v < kVariants[kernel]; ++v) {
            set_entry(kernel, cls, v);
            if ((st = run()) != BOBA_OK) break;
            if (count_diff(perm_out, rperm, n, dcnt, s) != 0 ||
                count_diff(src_out, rso, m, dcnt, s) != 0 ||
                count_diff(dst_out, rdo, m, dcnt, s) != 0) {
                continue;               // a variant that differs is never chosen
            }
            const double t = time_ms(run, reps, s);
            if (t < best_ms) { best_ms = t; best = v; }
        }
        set_entry(kernel, cls, best);
        if (chosen) chosen[k] = best;
    }
done:
    cudaFree(ref);
    cudaFree(dcnt);
    if (cudaGetLastError() != cudaSuccess) return BOBA_ERR_CUDA;
    return st;
}

extern "C" boba_status_t boba_tune_batched(const int32_t *src, const int32_t *dst,
                                           const int64_t *edge_off, const int64_t *vert_off,
                                           int64_t G, int64_t max_m, int64_t max_n,
                                           int64_t total_m, int64_t total_n, int32_t *perm_out,
                                           int32_t *src_out, int32_t *dst_out, void *ws,
                                           size_t ws_bytes, int reps, int *chosen, void *stream_)
{
    if (reps < 1 || total_m <= 0 || total_n <= 0) return BOBA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    const int cls = size_class(total_m);
    void *ref = nullptr;
    unsigned long long *dcnt = nullptr;
    if (cudaMalloc(&ref, (size_t)(2 * total_m + total_n) * 4) != cudaSuccess ||
        cudaMalloc(&dcnt, 8) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ref) cudaFree(ref);
        return BOBA_ERR_CUDA;
    }
    int32_t *rperm = static_cast<int32_t *>(ref), *rso = rperm + total_n, *rdo = rso + total_m;
    auto run = [&] {
        return boba_reorder_batched(src, dst, edge_off, vert_off, G, max_m, max_n, total_m,
                                    total_n, perm_out, src_out, dst_out, ws, ws_bytes, s);
    };
    boba_status_t st = BOBA_OK;
    int best = 0;
    double best_ms = 1e30;
    for (int v = 0; v < kVariants[kTuneBatched]; ++v) {
        set_entry(kTuneBatched, cls, v);
        if (boba_reorder_batched_workspace_bytes(G, max_m, max_n, total_m, total_n) > ws_bytes)
            continue;                   // this schedule needs more scratch than given
        if ((st = run()) != BOBA_OK) break;
        if (v == 0) {
            cudaMemcpyAsync(rperm, perm_out, 4 * (size_t)total_n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(rso, src_out, 4 * (size_t)total_m, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(rdo, dst_out, 4 * (size_t)total_m, cudaMemcpyDeviceToDevice, s);
        } else if (count_diff(perm_out, rperm, total_n, dcnt, s) != 0 ||
                   count_diff(src_out, rso, total_m, dcnt, s) != 0 ||
                   count_diff(dst_out, rdo, total_m, dcnt, s) != 0) {
            continue;
        }
        const double t = time_ms(run, reps, s);
        if (t < best_ms) { best_ms = t; best = v; }
    }
    set_entry(kTuneBatched, cls, best);
    if (chosen) chosen[0] = best;
    cudaFree(ref);
    cudaFree(dcnt);
    if (cudaGetLastError() != cudaSuccess) return BOBA_ERR_CUDA;
    return st;
}

extern "C" boba_status_t boba_tune_spmv(const int64_t *row_ptr, const int32_t *col, const float *val,
                                        const float *x, float *y, int64_t n_rows, int64_t nnz,
                                        void *ws, size_t ws_bytes, int reps, int *chosen,
                                        void *stream_)
{
    if (reps < 1 || n_rows <= 0) return BOBA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    const int cls = size_class(nnz);
    // variant 0's product is the reference: a variant further than
    // kSpmvTuneRelL2 from it (relative L2) is never chosen
    float *ref = nullptr;
    double *dsums = nullptr;
    if (cudaMalloc(&ref, (size_t)n_rows * 4) != cudaSuccess ||
        cudaMalloc(&dsums, 2 * sizeof(double)) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ref) cudaFree(ref);
        return BOBA_ERR_CUDA;
    }
    int best = 0;
    double best_ms = 1e30;
    boba_status_t st = BOBA_OK;
    for (int v = 0; v < kVariants[kTuneSpmv]; ++v) {
        set_entry(kTuneSpmv, cls, v);
        auto run = [&] { return boba_spmv_csr(row_ptr, col, val, x, y, n_rows, nnz, ws, ws_bytes, s); };
        if ((st = run()) != BOBA_OK) break;
        if (v == 0) {
            cudaMemcpyAsync(ref, y, (size_t)n_rows * 4, cudaMemcpyDeviceToDevice, s);
        } else {
            const double e = rel_l2(y, ref, n_rows, dsums, s);
            if (e < 0.0 || e > kSpmvTuneRelL2) continue;
        }
        const double t = time_ms(run, reps, s);
        if (t < best_ms) { best_ms = t; best = v; }
    }
    set_entry(kTuneSpmv, cls, best);
    if (chosen) chosen[0] = best;
    cudaFree(ref);
    cudaFree(dsums);
    if (cudaGetLastError() != cudaSuccess) return BOBA_ERR_CUDA;
    return st;
}

extern "C" boba_status_t boba_tune_csr(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                       int64_t *row_ptr, int32_t *col_out, float *val_out, void *ws,
                                       size_t ws_bytes, int reps, int *chosen, void *stream_)
{
    if (reps < 1 || m <= 0 || n <= 0) return BOBA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    const int cls = size_class(m);
    void *ref = nullptr;
    unsigned long long *dcnt = nullptr;
    if (cudaMalloc(&ref, (size_t)m * 8 + (size_t)(n + 1) * 8) != cudaSuccess ||
        cudaMalloc(&dcnt, 8) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ref) cudaFree(ref);
        return BOBA_ERR_CUDA;
    }
    int32_t *rcol = static_cast<int32_t *>(ref);
    float *rval = reinterpret_cast<float *>(rcol + m);
    int64_t *rrp = reinterpret_cast<int64_t *>(rval + m);
    auto run = [&] {
        return boba_coo_to_csr(src, dst, m, n, row_ptr, col_out, val_out, ws, ws_bytes, s);
    };
    boba_status_t st = BOBA_OK;
    int best = 0;
    double best_ms = 1e30;
    for (int v = 0; v < kVariants[kTuneCsr]; ++v) {
        set_entry(kTuneCsr, cls, v);
        if ((st = run()) != BOBA_OK) break;
        if (v == 0) {
            cudaMemcpyAsync(rcol, col_out, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(rval, val_out, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(rrp, row_ptr, 8 * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s);
        } else if (count_diff(col_out, rcol, m, dcnt, s) != 0 ||
                   count_diff(val_out, rval, m, dcnt, s) != 0 ||
                   count_diff(row_ptr, rrp, 2 * (n + 1), dcnt, s) != 0) {
            continue;
        }
        const double t = time_ms(run, reps, s);
        if (t < best_ms) { best_ms = t; best = v; }
    }
    set_entry(kTuneCsr, cls, best);
    if (chosen) chosen[0] = best;
    cudaFree(ref);
    cudaFree(dcnt);
    if (cudaGetLastError() != cudaSuccess) return BOBA_ERR_CUDA;
    return st;
}

extern "C" boba_status_t boba_tune_save(const char *path)
{
    if (!path) return BOBA_ERR_INVALID_ARG;
    const std::string name = dev_name();
    const int d = cur_dev();
    if (d < 0) return BOBA_ERR_CUDA;
    FILE *f = fopen(path, "w");
    if (!f) return BOBA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tmu);
    init_table();
    fprintf(f, "# boba autotune: gpu kernel size_class variant\n");
    for (int k = 0; k < kTuneKernels; ++k)
        for (int c = 0; c < kClasses; ++c)
            if (g_table[d][k][c] >= 0)
                fprintf(f, "%s %s %d %d\n", name.c_str(), kNames[k], c, (int)g_table[d][k][c]);
    fclose(f);
    return BOBA_OK;
}

extern "C" boba_status_t boba_tune_load(const char *path)
{
    if (!path) return BOBA_ERR_INVALID_ARG;
    const std::string name = dev_name();
    FILE *f = fopen(path, "r");
    if (!f) return BOBA_ERR_INVALID_ARG;
    char line[512];
    int loaded = 0;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        char gpu[256], kern[64];
        int c = -1, v = -1;
        if (sscanf(line, "%255s %63s %d %d", gpu, kern, &c, &v) != 4) continue;
        if (name != gpu) continue;
        for (int k = 0; k < kTuneKernels; ++k)
            if (strcmp(kern, kNames[k]) == 0 && c >= 0 && c < kClasses && v >= 0 && v < kVariants[k]) {
                set_entry(k, c, v);
                ++loaded;
            }
    }
    fclose(f);
    return loaded >= 0 ? BOBA_OK : BOBA_ERR_INVALID_ARG;
}
