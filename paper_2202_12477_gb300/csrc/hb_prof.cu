// Kernel launch counter and optional per-kernel timing with CUDA events.
//
// Every launcher of the library counts its launches. When timing is enabled,
// launchers also bracket their kernel with a pair of events recorded on the
// launch stream; hb_profile_read sums the elapsed times per kernel name.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hb_internal.h"

namespace {

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_prof_on{0};

struct prof_rec {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used;
};
std::mutex g_mu;
std::map<std::string, prof_rec> g_recs;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pool;

std::pair<cudaEvent_t, cudaEvent_t> take_pair()
{
    if (!g_pool.empty()) {
        auto p = g_pool.back();
        g_pool.pop_back();
        return p;
    }
    std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
    cudaEventCreate(&p.first);
    cudaEventCreate(&p.second);
    return p;
}

}  // namespace

void hb_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void hb_count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
bool hb_profiling_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

hb_prof_scope::hb_prof_scope(const char *name, cudaStream_t s) : stream(s), stop(nullptr)
{
    hb_count_launch();
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto p = take_pair();
    if (!p.first || !p.second) return;
    g_recs[name].used.push_back(p);
    cudaEventRecord(p.first, s);
    stop = p.second;
}

hb_prof_scope::~hb_prof_scope()
{
    if (stop) cudaEventRecord(stop, stream);
}

extern "C" unsigned long long hb_kernel_launches(void) { return g_launches.load(); }

extern "C" hb_status hb_profile_enable(int on)
{
    g_prof_on.store(on ? 1 : 0);
    return HB_OK;
}

extern "C" hb_status hb_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_recs)
        for (auto &p : kv.second.used) g_pool.push_back(p);
    g_recs.clear();
    return HB_OK;
}

extern "C" hb_status hb_profile_read(const char *name, double *total_ms, long long *launches)
{
    hb_clear_error();
    if (!name || !total_ms || !launches) { hb_set_error("null argument"); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    *total_ms = 0.0;
    *launches = 0;
    auto it = g_recs.find(name);
    if (it == g_recs.end()) return HB_OK;
    for (auto &p : it->second.used) {
        HB_TRY_CUDA(cudaEventSynchronize(p.second));
        float ms = 0.f;
        HB_TRY_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
        *total_ms += ms;
        *launches += 1;
    }
    return HB_OK;
}
