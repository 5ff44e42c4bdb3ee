// Serving runtime: requests (a COO graph, an x vector) arrive over time; each
// is reordered with BOBA, converted to CSR and multiplied by x a fixed number
// of times (Alg. 3), and y (plus, optionally, the permutation) is copied back.
//
// Continuous batching under an HBM budget:
//   * one device pool of `budget` bytes is allocated when the server is
//     created; requests are placed in it by a first-fit allocator, never by
//     cudaMalloc on the request path;
//   * a scheduler thread admits waiting requests in arrival order whenever a
//     slot is free and the pool has room, so requests that arrive while others
//     are on the GPU join as soon as memory frees up;
//   * the requests admitted together form a wave (up to kWaveEdges edges):
//     their graphs are copied in on a copy stream, packed, and reordered by
//     one boba_reorder_batched launch, so the next wave's copies overlap this
//     wave's compute; each request then runs its
//     CSR build, SpMV iterations and copy back on its own stream, so waves and
//     requests overlap on the device and a small request is not held back by
//     a large one;
//   * a request's memory is returned when the last request of its wave is done.
// Every kernel computes each request independently of the others, so a
// request's results are the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "host.hpp"

namespace boba {
namespace {

using Clock = std::chrono::steady_clock;

// Edges above which a wave takes no further request (a request larger than
// this forms a wave of its own).
constexpr int64_t kWaveEdges = 1ll << 26;

// First-fit allocator over one device region (host bookkeeping only).
class DevicePool {
public:
    bool init(size_t bytes)
    {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    ~DevicePool()
    {
        if (base_) cudaFree(base_);
    }
    // Returns an offset, or SIZE_MAX if no free range fits.
    size_t alloc(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                sizes_[off] = bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }
    char *at(size_t off) const { return static_cast<char *>(base_) + off; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;     // offset -> length
    std::map<size_t, size_t> sizes_;    // allocated offset -> length
};

struct Wave;

struct Request {
    int64_t id = 0;
    const int32_t *src_h = nullptr, *dst_h = nullptr;
    const float *x_h = nullptr;
    float *y_h = nullptr;
    int32_t *perm_h = nullptr;
    int64_t m = 0, n = 0;
    Clock::time_point arrival, admitted, done_at;
    std::shared_ptr<Wave> wave;
    size_t packed_e = 0, packed_v = 0;       // offsets inside the wave's packed arrays
    // per-request device arrays inside the wave block
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    float *val = nullptr, *x = nullptr, *y = nullptr;
    void *csr_ws = nullptr, *spmv_ws = nullptr;
    size_t csr_ws_bytes = 0, spmv_ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t started = nullptr;           // its stream reached its work (after the wave's reorder)
    cudaEvent_t done = nullptr;
    boba_status_t status = BOBA_OK;
};

struct Wave {
    size_t block_off = SIZE_MAX;
    int remaining = 0;
    std::vector<int64_t> eoff, voff;         // host copies (kept alive for the async copies)
};

// Device bytes of one request's own arrays (CSR, x, y, workspaces).
size_t request_bytes(int64_t m, int64_t n)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(8 * (size_t)(n + 1)) + al(4 * (size_t)m) * 2 + al(4 * (size_t)n) * 2 +
           al(boba_coo_to_csr_workspace_bytes(m, n)) + al(boba_spmv_workspace_bytes(n, m));
}

// Device bytes of a wave: packed COO in/out, perm, offsets, batched workspace,
// plus every request's own arrays.
size_t wave_bytes(const std::vector<Request *> &rs)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    int64_t tm = 0, tn = 0, mm = 0, mn = 0;
    size_t own = 0;
    for (const Request *r : rs) {
        tm += r->m;
        tn += r->n;
        mm = std::max(mm, r->m);
        mn = std::max(mn, r->n);
        own += request_bytes(r->m, r->n);
    }
    const int64_t G = (int64_t)rs.size();
    return al(4 * (size_t)tm) * 4 + al(4 * (size_t)tn) + al(8 * (size_t)(G + 1)) * 2 +
           al(boba_reorder_batched_workspace_bytes(G, mm, mn, tm, tn)) + own;
}

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0;
    int max_active = 0, spmv_iters = 0;
    DevicePool pool;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::list<Request *> active;
    std::vector<Request *> finished;          // not yet returned by poll
    std::vector<double> latencies_ms;
    std::vector<double> queue_ms, service_ms;     // arrival -> admission, admission -> done
    std::vector<std::pair<float, float>> device_spans;   // [start, end] ms since `epoch`
    cudaEvent_t epoch = nullptr;              // reference point of the device spans
    size_t peak_active = 0;                   // most requests admitted at once
    int64_t joined_busy = 0;                  // requests admitted while others were active
    int64_t next_id = 0, edges_done = 0, requests_done = 0;
    Clock::time_point first_arrival, last_done;
    bool any_arrival = false;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    cudaStream_t wave_stream = nullptr;
    cudaStream_t copy_stream = nullptr;       // a wave's input copies, ahead of its reorder
    boba_status_t error = BOBA_OK;

    void run();
    bool launch_wave(std::vector<Request *> &wave);
};

bool Server::launch_wave(std::vector<Request *> &rs)
{
    auto W = std::make_shared<Wave>();
    const size_t bytes = wave_bytes(rs);
    W->block_off = pool.alloc(bytes);
    if (W->block_off == SIZE_MAX) return false;
    W->remaining = (int)rs.size();
    int64_t tm = 0, tn = 0, mm = 0, mn = 0;
    W->eoff.assign(1, 0);
    W->voff.assign(1, 0);
    for (Request *r : rs) {
        r->packed_e = (size_t)tm;
        r->packed_v = (size_t)tn;
        tm += r->m;
        tn += r->n;
        mm = std::max(mm, r->m);
        mn = std::max(mn, r->n);
        W->eoff.push_back(tm);
        W->voff.push_back(tn);
    }
    const int64_t G = (int64_t)rs.size();
    char *p = pool.at(W->block_off);
    Carve c;
    int32_t *src = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)tm));
    int32_t *dst = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)tm));
    int32_t *so = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)tm));
    int32_t *dout = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)tm));
    int32_t *perm = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)tn));
    int64_t *eo = reinterpret_cast<int64_t *>(p + c.take(8 * (size_t)(G + 1)));
    int64_t *vo = reinterpret_cast<int64_t *>(p + c.take(8 * (size_t)(G + 1)));
    const size_t bws = boba_reorder_batched_workspace_bytes(G, mm, mn, tm, tn);
    void *bw = p + c.take(bws);
    for (Request *r : rs) {
        r->row_ptr = reinterpret_cast<int64_t *>(p + c.take(8 * (size_t)(r->n + 1)));
        r->col = reinterpret_cast<int32_t *>(p + c.take(4 * (size_t)r->m));
        r->val = reinterpret_cast<float *>(p + c.take(4 * (size_t)r->m));
        r->x = reinterpret_cast<float *>(p + c.take(4 * (size_t)r->n));
        r->y = reinterpret_cast<float *>(p + c.take(4 * (size_t)r->n));
        r->csr_ws_bytes = boba_coo_to_csr_workspace_bytes(r->m, r->n);
        r->csr_ws = p + c.take(r->csr_ws_bytes);
        r->spmv_ws_bytes = boba_spmv_workspace_bytes(r->n, r->m);
        r->spmv_ws = p + c.take(r->spmv_ws_bytes);
        r->wave = W;
    }
    // inputs of the wave, packed, on the copy stream: the next wave's copies
    // then run while this wave's reorder and its requests compute
    cudaStream_t cs = copy_stream;
    for (Request *r : rs) {
        if (r->m > 0) {
            cudaMemcpyAsync(src + r->packed_e, r->src_h, 4 * (size_t)r->m, cudaMemcpyHostToDevice, cs);
            cudaMemcpyAsync(dst + r->packed_e, r->dst_h, 4 * (size_t)r->m, cudaMemcpyHostToDevice, cs);
        }
    }
    cudaMemcpyAsync(eo, W->eoff.data(), 8 * (size_t)(G + 1), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(vo, W->voff.data(), 8 * (size_t)(G + 1), cudaMemcpyHostToDevice, cs);
    cudaEvent_t landed;
    cudaEventCreateWithFlags(&landed, cudaEventDisableTiming);
    cudaEventRecord(landed, cs);
    cudaStream_t ws = wave_stream;
    cudaStreamWaitEvent(ws, landed, 0);
    cudaEventDestroy(landed);        // released once its work completes
    boba_status_t st = boba_reorder_batched(src, dst, eo, vo, G, mm, mn, tm, tn, perm, so, dout,
                                            bw, bws, ws);
    cudaEvent_t reordered;
    cudaEventCreateWithFlags(&reordered, cudaEventDisableTiming);
    cudaEventRecord(reordered, ws);
    for (Request *r : rs) {
        r->status = st;
        r->stream = streams[next_stream++ % streams.size()];
        cudaStreamWaitEvent(r->stream, reordered, 0);
        cudaEventCreate(&r->started);
        cudaEventRecord(r->started, r->stream);
        if (r->x_h) cudaMemcpyAsync(r->x, r->x_h, 4 * (size_t)r->n, cudaMemcpyHostToDevice, r->stream);
        if (st == BOBA_OK)
            st = boba_coo_to_csr(so + r->packed_e, dout + r->packed_e, r->m, r->n, r->row_ptr,
                                 r->col, r->val, r->csr_ws, r->csr_ws_bytes, r->stream);
        for (int it = 0; it < spmv_iters && st == BOBA_OK; ++it)
            st = boba_spmv_csr(r->row_ptr, r->col, r->val, r->x, r->y, r->n, r->m, r->spmv_ws,
                               r->spmv_ws_bytes, r->stream);
        if (r->y_h) cudaMemcpyAsync(r->y_h, r->y, 4 * (size_t)r->n, cudaMemcpyDeviceToHost, r->stream);
        if (r->perm_h)
            cudaMemcpyAsync(r->perm_h, perm + r->packed_v, 4 * (size_t)r->n, cudaMemcpyDeviceToHost,
                            r->stream);
        r->status = st;
        cudaEventCreate(&r->done);
        cudaEventRecord(r->done, r->stream);
    }
    cudaEventDestroy(reordered);     // released once its work completes
    if (cudaGetLastError() != cudaSuccess) error = BOBA_ERR_CUDA;
    return true;
}

void Server::run()
{
    cudaSetDevice(device);
    while (true) {
        std::vector<Request *> wave;
        {
            std::unique_lock<std::mutex> lk(mu);
            // completions
            for (auto it = active.begin(); it != active.end();) {
                Request *r = *it;
                const cudaError_t q = cudaEventQuery(r->done);
                if (q == cudaErrorNotReady) { ++it; continue; }
                if (q != cudaSuccess) { r->status = BOBA_ERR_CUDA; (void)cudaGetLastError(); }
                r->done_at = Clock::now();
                float t0 = 0.f, t1 = 0.f;
                if (cudaEventElapsedTime(&t0, epoch, r->started) == cudaSuccess &&
                    cudaEventElapsedTime(&t1, epoch, r->done) == cudaSuccess)
                    device_spans.emplace_back(t0, t1);
                else
                    (void)cudaGetLastError();
                cudaEventDestroy(r->started);
                cudaEventDestroy(r->done);
                r->started = r->done = nullptr;
                latencies_ms.push_back(
                    std::chrono::duration<double, std::milli>(r->done_at - r->arrival).count());
                queue_ms.push_back(
                    std::chrono::duration<double, std::milli>(r->admitted - r->arrival).count());
                service_ms.push_back(
                    std::chrono::duration<double, std::milli>(r->done_at - r->admitted).count());
                edges_done += r->m;
                requests_done += 1;
                last_done = r->done_at;
                if (--r->wave->remaining == 0) pool.release(r->wave->block_off);
                r->wave.reset();
                finished.push_back(r);
                it = active.erase(it);
            }
            // admission, in arrival order, while slots and memory allow; a
            // wave stops growing at kWaveEdges edges so that the next one's
            // copies overlap its compute (it always takes one request)
            int64_t wave_edges = 0;
            while (!pending.empty() && (int)(active.size() + wave.size()) < max_active &&
                   (wave.empty() || wave_edges + pending.front()->m <= kWaveEdges)) {
                wave.push_back(pending.front());
                if (wave_bytes(wave) + pool.used() > pool.size()) {
                    wave.pop_back();
                    break;
                }
                wave_edges += pending.front()->m;
                pending.pop_front();
            }
            if (!wave.empty()) {
                if (!launch_wave(wave)) {            // fragmentation: retry later
                    for (auto it = wave.rbegin(); it != wave.rend(); ++it) pending.push_front(*it);
                    wave.clear();
                } else {
                    const Clock::time_point now = Clock::now();
                    if (!active.empty()) joined_busy += (int64_t)wave.size();
                    for (Request *r : wave) {
                        r->admitted = now;
                        active.push_back(r);
                    }
                    peak_active = std::max(peak_active, active.size());
                }
            }
            if (stop.load() && pending.empty() && active.empty()) break;
            if (wave.empty())
                cv.wait_for(lk, std::chrono::microseconds(active.empty() ? 500 : 20));
        }
    }
}

}  // namespace boba

using namespace boba;

extern "C" {

typedef struct boba_server boba_server_t;

boba_server_t *boba_server_create(size_t hbm_budget_bytes, int max_active, int spmv_iters,
                                  int n_streams)
{
    if (hbm_budget_bytes < (1u << 20) || max_active < 1 || spmv_iters < 0 || n_streams < 1)
        return nullptr;
    auto *S = new Server();
    if (cudaGetDevice(&S->device) != cudaSuccess || !S->pool.init(hbm_budget_bytes)) {
        (void)cudaGetLastError();
        delete S;
        return nullptr;
    }
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->spmv_iters = spmv_iters;
    for (int i = 0; i < n_streams; ++i) {
        cudaStream_t s;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        S->streams.push_back(s);
    }
    cudaStreamCreateWithFlags(&S->wave_stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    cudaEventCreate(&S->epoch);
    cudaEventRecord(S->epoch, S->wave_stream);
    S->worker = std::thread([S] { S->run(); });
    return reinterpret_cast<boba_server_t *>(S);
}

int64_t boba_server_submit(boba_server_t *h, const int32_t *src_host, const int32_t *dst_host,
                           int64_t m, int64_t n, const float *x_host, float *y_host,
                           int32_t *perm_host)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S || m < 0 || n < 1 || m > kMaxSize || n > kMaxSize) return -1;
    if (m > 0 && (src_host == nullptr || dst_host == nullptr)) return -1;
    std::vector<Request *> one;
    Request probe;
    probe.m = m;
    probe.n = n;
    one.push_back(&probe);
    if (wave_bytes(one) > S->budget) return -2;          // can never be admitted
    auto *r = new Request();
    r->src_h = src_host;
    r->dst_h = dst_host;
    r->x_h = x_host;
    r->y_h = y_host;
    r->perm_h = perm_host;
    r->m = m;
    r->n = n;
    r->arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        if (!S->any_arrival) { S->first_arrival = r->arrival; S->any_arrival = true; }
        S->pending.push_back(r);
    }
    S->cv.notify_one();
    return r->id;
}

int boba_server_poll(boba_server_t *h, int64_t *ids, double *latency_ms, int *status, int cap)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S || cap < 0) return -1;
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    while (k < cap && !S->finished.empty()) {
        Request *r = S->finished.back();
        S->finished.pop_back();
        if (ids) ids[k] = r->id;
        if (latency_ms)
            latency_ms[k] = std::chrono::duration<double, std::milli>(r->done_at - r->arrival).count();
        if (status) status[k] = (int)r->status;
        delete r;
        ++k;
    }
    return k;
}

boba_status_t boba_server_cancel(boba_server_t *h, int64_t id)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S) return BOBA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
        if ((*it)->id != id) continue;
        delete *it;                 // not admitted: nothing of it is on the device
        S->pending.erase(it);
        return BOBA_OK;
    }
    return BOBA_ERR_INVALID_ARG;    // unknown, or already admitted
}

boba_status_t boba_server_drain(boba_server_t *h)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S) return BOBA_ERR_INVALID_ARG;
    while (true) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->pending.empty() && S->active.empty()) break;
        }
        S->cv.notify_one();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    return S->error;
}

int boba_server_stats(boba_server_t *h, double *out, int cap)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S || !out || cap < 7) return -1;
    std::lock_guard<std::mutex> lk(S->mu);
    auto pct_of = [](std::vector<double> v, double q) {
        if (v.empty()) return 0.0;
        std::sort(v.begin(), v.end());
        size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
        return v[std::min(i, v.size() - 1)];
    };
    auto pct = [&](double q) { return pct_of(S->latencies_ms, q); };
    const double span =
        S->any_arrival && S->requests_done > 0
            ? std::chrono::duration<double>(S->last_done - S->first_arrival).count()
            : 0.0;
    out[0] = pct(0.50);
    out[1] = pct(0.99);
    out[2] = span > 0 ? (double)S->edges_done / span / 1e9 : 0.0;   // Gedges/s
    out[3] = (double)S->requests_done;
    out[4] = (double)S->edges_done;
    out[5] = (double)S->pool.peak();
    out[6] = span;
    if (cap < 13) return 7;
    // most requests whose device work overlapped: a sweep over the spans
    std::vector<std::pair<float, int>> ev;
    for (const auto &sp : S->device_spans) {
        ev.emplace_back(sp.first, 1);
        ev.emplace_back(sp.second, -1);
    }
    std::sort(ev.begin(), ev.end());          // an end before a start at the same instant
    int cur = 0, best = 0;
    for (const auto &e : ev) best = std::max(best, cur += e.second);
    out[7] = (double)S->peak_active;
    out[8] = (double)S->joined_busy;
    out[9] = (double)best;
    out[10] = pct_of(S->queue_ms, 0.50);
    out[11] = pct_of(S->queue_ms, 0.99);
    out[12] = pct_of(S->service_ms, 0.99);
    return 13;
}

void boba_server_destroy(boba_server_t *h)
{
    auto *S = reinterpret_cast<Server *>(h);
    if (!S) return;
    boba_server_drain(h);
    S->stop.store(true);
    S->cv.notify_one();
    if (S->worker.joinable()) S->worker.join();
    for (Request *r : S->finished) delete r;
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    cudaStreamDestroy(S->wave_stream);
    cudaStreamDestroy(S->copy_stream);
    cudaEventDestroy(S->epoch);
    delete S;
}

}  // extern "C"
