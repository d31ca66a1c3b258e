// profile.cu -- launch counter and CUDA-event timing of the hot kernels.
#include <atomic>
#include <mutex>
#include <vector>

#include "hd_internal.cuh"

namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};

struct event_pair {
    cudaEvent_t a = nullptr, b = nullptr;
};

struct prof_state {
    std::mutex mu;
    std::vector<event_pair> pool;                       // reusable pairs
    std::vector<event_pair> recorded[HD_KERNEL_KINDS];  // waiting to be collected
} g_prof;

}  // namespace

void hd_count_launches(uint32_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

hd_prof_scope::hd_prof_scope(hd_kernel_kind k, cudaStream_t st) : kind(k), s(st)
{
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    event_pair e;
    {
        std::lock_guard<std::mutex> g(g_prof.mu);
        if (!g_prof.pool.empty()) {
            e = g_prof.pool.back();
            g_prof.pool.pop_back();
        }
    }
    if (!e.a && (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess)) return;
    // the stop event is recorded by the destructor, after the launch
    cudaEventRecord(e.a, s);
    ev_a = e.a;
    ev_b = e.b;
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.recorded[kind].push_back(e);
}

hd_prof_scope::~hd_prof_scope()
{
    if (ev_b) cudaEventRecord((cudaEvent_t)ev_b, s);
}

extern "C" {

hd_status hd_profile_enable(int on)
{
    g_enabled.store(on ? 1 : 0);
    return HD_OK;
}

hd_status hd_profile_collect(hd_kernel_kind kind, double *total_ms, uint32_t *launches)
{
    if ((int)kind < 0 || (int)kind >= HD_KERNEL_KINDS)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_profile_collect: bad kernel kind");
    std::vector<event_pair> ev;
    {
        std::lock_guard<std::mutex> g(g_prof.mu);
        ev.swap(g_prof.recorded[kind]);
    }
    double tot = 0.0;
    for (auto &e : ev) {
        float ms = 0.f;
        cudaEventSynchronize(e.b);
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) tot += ms;
    }
    {
        std::lock_guard<std::mutex> g(g_prof.mu);
        g_prof.pool.insert(g_prof.pool.end(), ev.begin(), ev.end());
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (uint32_t)ev.size();
    return HD_OK;
}

uint64_t hd_launch_count(void) { return g_launches.load(); }

}  // extern "C"
