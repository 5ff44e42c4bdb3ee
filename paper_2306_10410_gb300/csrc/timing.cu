// Per-kernel timing with CUDA events recorded on the launching stream.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host.hpp"

namespace boba {

namespace {
std::atomic<bool> g_on{false};
std::mutex g_mu;
struct Pending {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
struct Total {
    std::string name;
    double ms = 0;
    int64_t launches = 0;
};
std::vector<Total> g_totals;

cudaEvent_t get_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

bool timing_on() { return g_on.load(std::memory_order_relaxed); }

void timing_begin(const char *name, cudaStream_t s, int *slot)
{
    std::lock_guard<std::mutex> lk(g_mu);
    Pending p;
    p.name = name;
    p.a = get_event();
    p.b = get_event();
    if (!p.a || !p.b || cudaEventRecord(p.a, s) != cudaSuccess) {
        (void)cudaGetLastError();
        *slot = -1;
        return;
    }
    g_pending.push_back(p);
    *slot = (int)g_pending.size() - 1;
}

void timing_end(int slot, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < 0 || slot >= (int)g_pending.size()) return;
    if (cudaEventRecord(g_pending[slot].b, s) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace boba

using namespace boba;

extern "C" void boba_timing_enable(int on) { g_on.store(on != 0); }

extern "C" int boba_timing_collect(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = 0;
    for (Pending &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = -1;
        } else {
            Total *t = nullptr;
            for (Total &x : g_totals)
                if (x.name == p.name) t = &x;
            if (!t) {
                g_totals.push_back(Total{p.name, 0.0, 0});
                t = &g_totals.back();
            }
            t->ms += ms;
            t->launches += 1;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
    return rc < 0 ? -1 : (int)g_totals.size();
}

extern "C" const char *boba_timing_name(int i)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return (i >= 0 && i < (int)g_totals.size()) ? g_totals[i].name.c_str() : "";
}

extern "C" double boba_timing_total_ms(int i)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return (i >= 0 && i < (int)g_totals.size()) ? g_totals[i].ms : 0.0;
}

extern "C" int64_t boba_timing_launches(int i)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return (i >= 0 && i < (int)g_totals.size()) ? g_totals[i].launches : 0;
}

extern "C" void boba_timing_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (Pending &p : g_pending) {
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
    g_totals.clear();
}
