// Launch accounting: every kernel launch of the library goes through
// record_launch(); with profiling on, each launch is bracketed by CUDA events
// on its own stream so per-kernel device time can be read back.
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

static std::mutex g_prof_mu;
static unsigned long long g_launches = 0;
static bool g_prof_on = false;

struct ProfEntry {
    std::string name;
    cudaEvent_t a, b;
};
static std::vector<ProfEntry> g_pending;

struct ProfTotal {
    std::string name;
    unsigned long long launches = 0;
    double ms = 0;
};
static std::vector<ProfTotal> g_totals;

// Timing events are reused (created once, returned to the pool when their
// times have been read), so a timed launch costs two event records and no
// event creation.
static std::vector<cudaEvent_t> g_event_pool;

static bool take_event(cudaEvent_t* e) {  // caller holds g_prof_mu
    if (!g_event_pool.empty()) {
        *e = g_event_pool.back();
        g_event_pool.pop_back();
        return true;
    }
    return cudaEventCreate(e) == cudaSuccess;
}

LaunchScope::LaunchScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
    bool take = false;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        ++g_launches;
        take = g_prof_on && take_event((cudaEvent_t*)&a_) && take_event((cudaEvent_t*)&b_);
    }
    if (take) {
        cudaEventRecord((cudaEvent_t)a_, s_);
        timed_ = true;
    }
}

LaunchScope::~LaunchScope() {
    if (!timed_) return;
    cudaEventRecord((cudaEvent_t)b_, s_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back({name_, (cudaEvent_t)a_, (cudaEvent_t)b_});
}

static void drain_pending() {
    for (auto& e : g_pending) {
        float ms = 0;
        cudaEventSynchronize(e.b);
        cudaEventElapsedTime(&ms, e.a, e.b);
        g_event_pool.push_back(e.a);
        g_event_pool.push_back(e.b);
        ProfTotal* t = nullptr;
        for (auto& x : g_totals)
            if (x.name == e.name) t = &x;
        if (!t) {
            g_totals.push_back(ProfTotal{e.name});
            t = &g_totals.back();
        }
        t->launches += 1;
        t->ms += ms;
    }
    g_pending.clear();
}

}  // namespace dsg

using namespace dsg;

extern "C" {

void dsg_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
}

void dsg_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    g_totals.clear();
}

unsigned long long dsg_launch_count(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_launches;
}

/* Writes up to cap entries "name launches total_ms\n" into buf; returns the
 * number of kernels with timings. */
int dsg_profile_report(char* buf, size_t cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    size_t used = 0;
    if (buf && cap) buf[0] = 0;
    for (auto& t : g_totals) {
        if (!buf) break;
        int k = snprintf(buf + used, cap > used ? cap - used : 0, "%s %llu %.6f\n", t.name.c_str(), t.launches, t.ms);
        if (k < 0 || used + (size_t)k >= cap) break;
        used += (size_t)k;
    }
    return (int)g_totals.size();
}

}  // extern "C"
