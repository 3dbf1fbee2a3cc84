// Launch counter and per-kernel-class event timing (diagnostics API of hssnd.h).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace hssnd {

namespace {
struct Rec {
    cudaEvent_t a, b;
    int cls;
};
struct ClassStat {
    std::string name;
    double total_ms = 0.0;
    long launches = 0;
    double work = 0.0;
};
std::mutex g_mu;
std::atomic<long> g_launches{0};
bool g_on = false;
bool g_host_only = false;   // mode 2: host sections only, no events
std::vector<ClassStat> g_cls;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;

int class_of(const char *name) {
    for (size_t i = 0; i < g_cls.size(); ++i)
        if (g_cls[i].name == name) return (int)i;
    g_cls.push_back({name});
    return (int)g_cls.size() - 1;
}

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void drain_locked() {
    for (auto &r : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            g_cls[r.cls].total_ms += ms;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
}
}  // namespace

thread_local bool g_capturing = false;
thread_local bool g_rb_pending = false;
thread_local std::chrono::steady_clock::time_point g_rb_t;
thread_local double g_rb_gap_ms = 0.0;

void prof_mark_readback() {
    g_rb_pending = true;
    g_rb_t = std::chrono::steady_clock::now();
}
double prof_readback_gap_ms() { return g_rb_gap_ms; }

bool prof_enabled() { return g_on; }
void prof_set_capture(bool on) { g_capturing = on; }
void prof_add_launches(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(const char *name, cudaStream_t stream, double work) : cls(-1), s(stream), slot(-1) {
    if (g_capturing) return;
    if (g_rb_pending) {
        g_rb_pending = false;
        g_rb_gap_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g_rb_t).count();
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_on || g_host_only) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cls = class_of(name);
    g_cls[cls].launches++;
    g_cls[cls].work += work;
    Rec r{get_event(), get_event(), cls};
    cudaEventRecord(r.a, s);
    g_pending.push_back(r);
    slot = (int)g_pending.size() - 1;
    if (g_pending.size() > 4096) {
        // keep memory bounded: settle the finished records except ours
        Rec mine = g_pending.back();
        g_pending.pop_back();
        drain_locked();
        g_pending.push_back(mine);
        slot = 0;
    }
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, s);
}

HostScope::HostScope(const char *name) : cls(-1) {
    if (!g_on || g_capturing) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cls = class_of((std::string("host:") + name).c_str());
    t0 = std::chrono::steady_clock::now();
}

HostScope::~HostScope() {
    if (cls < 0) return;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lk(g_mu);
    g_cls[cls].total_ms += ms;
    g_cls[cls].launches++;
}

}  // namespace hssnd

using namespace hssnd;

extern "C" long hss_launch_count(void) { return g_launches.load(); }

extern "C" int hss_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!on) drain_locked();
    g_on = on != 0;
    g_host_only = on == 2;
    return HSS_OK;
}

extern "C" int hss_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    g_cls.clear();
    return HSS_OK;
}

extern "C" int hss_profile_read(int idx, char *name, int cap, double *total_ms, long *launches, double *work) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    if (idx < 0) return (int)g_cls.size();
    if (idx >= (int)g_cls.size()) {
        set_error("hss_profile_read: no such kernel class");
        return HSS_EINVAL;
    }
    const ClassStat &c = g_cls[idx];
    if (name && cap > 0) {
        std::strncpy(name, c.name.c_str(), cap - 1);
        name[cap - 1] = 0;
    }
    if (total_ms) *total_ms = c.total_ms;
    if (launches) *launches = c.launches;
    if (work) *work = c.work;
    return HSS_OK;
}
