// Launch accounting and optional per-kernel-class CUDA-event timing.
#pragma once
#include <chrono>
#include <cuda_runtime.h>

namespace hssnd {

// Every kernel launch of the library goes through one ProfScope: it counts
// the launch and, while profiling is enabled, brackets it with two events on
// the launching stream.  `work` is the algorithmic work the caller attributes
// to the launch (flops or bytes, by kernel class).
struct ProfScope {
    int cls;
    cudaStream_t s;
    int slot;
    ProfScope(const char *name, cudaStream_t stream, double work = 0.0);
    ~ProfScope();
};

// Host wall time of a named section of library host code (planning, uploads,
// launches), recorded as class "host:<name>" while profiling is enabled.
// Sections nest; each records its inclusive time.
struct HostScope {
    int cls;
    std::chrono::steady_clock::time_point t0;
    explicit HostScope(const char *name);
    ~HostScope();
};

// Host reaction time after a blocking read-back: mark_readback() notes the
// moment a read-back returns, the next kernel launch adds the time since then
// to a running total (the device has nothing queued meanwhile).
void prof_mark_readback();
double prof_readback_gap_ms();   // running total (ms)

bool prof_enabled();
void prof_set_capture(bool on);     // while a graph is being captured, scopes record nothing
void prof_add_launches(long n);     // kernels executed by a graph launch

}  // namespace hssnd

#define HSS_PROF(name, stream, ...) ::hssnd::ProfScope _prof_scope_(name, stream, ##__VA_ARGS__)
#define HSS_HOST_CAT2(a, b) a##b
#define HSS_HOST_CAT(a, b) HSS_HOST_CAT2(a, b)
#define HSS_HOST(name) ::hssnd::HostScope HSS_HOST_CAT(_host_scope_, __LINE__)(name)
