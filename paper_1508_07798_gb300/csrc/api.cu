// Error state, option defaults and small shared host utilities of libhssnd.
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "internal.h"

namespace hssnd {

static thread_local std::string g_last_error;

// Memory requests served by the library (diagnostics: hss_alloc_count).
static std::atomic<long> g_alloc_requests{0};
void count_alloc() { g_alloc_requests.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return HSS_ENOMEM;
    return HSS_ECUDA;
}

int DevBuf::alloc(size_t nbytes) {
    if (nbytes <= bytes && p) return HSS_OK;
    release();
    if (nbytes == 0) nbytes = 1;
    count_alloc();
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc of " + std::to_string(nbytes) + " bytes failed: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HSS_ENOMEM : HSS_ECUDA;
    }
    bytes = nbytes;
    return HSS_OK;
}

// Dynamic shared-memory limit of a kernel, set once per (device, kernel):
// the attribute belongs to the device context; the set is guarded for calls
// from several host threads, and the runtime's return code is passed on.
int device_sms() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
    return n;
}

cudaError_t func_smem_once(const void *func, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, func})) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({dev, func});
    return e;
}

// ---- scratch cache: device chunks and pinned buffers kept between calls
namespace {
struct ScratchCache {
    std::mutex mu;
    std::vector<std::pair<int, DevBuf>> dev;              // (device, chunk)
    std::vector<std::pair<void *, size_t>> pin;
    size_t dev_bytes = 0, pin_bytes = 0;
};
ScratchCache &cache() {
    static ScratchCache *c = new ScratchCache();   // never destroyed: no CUDA calls at process exit
    return *c;
}
constexpr size_t CACHE_DEV_MAX = (size_t)8 << 30;
constexpr size_t CACHE_PIN_MAX = (size_t)512 << 20;
int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}
}  // namespace

int scratch_cache_take_device(size_t min_bytes, size_t want_bytes, DevBuf &out) {
    count_alloc();
    const int d = current_device();
    {
        std::lock_guard<std::mutex> lk(cache().mu);
        auto &v = cache().dev;
        int best = -1;
        for (int k = 0; k < (int)v.size(); ++k)
            if (v[k].first == d && v[k].second.bytes >= min_bytes &&
                (best < 0 || v[k].second.bytes < v[best].second.bytes))
                best = k;
        if (best >= 0) {
            out = std::move(v[best].second);
            cache().dev_bytes -= out.bytes;
            v.erase(v.begin() + best);
            return HSS_OK;
        }
    }
    return out.alloc(want_bytes);
}

void scratch_cache_give_device(DevBuf &&b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> lk(cache().mu);
    if (cache().dev_bytes + b.bytes > CACHE_DEV_MAX) {
        b.release();
        return;
    }
    cache().dev_bytes += b.bytes;
    cache().dev.emplace_back(current_device(), std::move(b));
}

void *scratch_cache_take_pinned(size_t min_bytes, size_t want_bytes, size_t &got) {
    count_alloc();
    {
        std::lock_guard<std::mutex> lk(cache().mu);
        auto &v = cache().pin;
        int best = -1;
        for (int k = 0; k < (int)v.size(); ++k)
            if (v[k].second >= min_bytes && (best < 0 || v[k].second < v[best].second)) best = k;
        if (best >= 0) {
            void *p = v[best].first;
            got = v[best].second;
            cache().pin_bytes -= got;
            v.erase(v.begin() + best);
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, want_bytes) != cudaSuccess) {
        cudaGetLastError();
        got = 0;
        return nullptr;
    }
    got = want_bytes;
    return p;
}

void scratch_cache_give_pinned(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(cache().mu);
    if (cache().pin_bytes + bytes > CACHE_PIN_MAX) {
        cudaFreeHost(p);
        return;
    }
    cache().pin_bytes += bytes;
    cache().pin.emplace_back(p, bytes);
}

Work::~Work() {
    cudaStreamSynchronize(s);
    for (auto &c : chunks) scratch_cache_give_device(std::move(c));
    chunks.clear();
    if (hpin) scratch_cache_give_pinned(hpin, hcap);
    for (size_t k = 0; k < old_pins.size(); ++k) scratch_cache_give_pinned(old_pins[k], old_sizes[k]);
}

int Work::dalloc_bytes(size_t bytes, void **out) {
    count_alloc();
    bytes = (bytes + 255) & ~(size_t)255;
    while (ci < chunks.size() && cur + bytes > chunks[ci].bytes) {
        ++ci;
        cur = 0;
    }
    if (ci >= chunks.size()) {
        size_t want = std::max(bytes, std::max((size_t)(16u << 20), chunks.empty() ? 0 : 2 * chunks.back().bytes));
        DevBuf b;
        int rc = scratch_cache_take_device(bytes, want, b);
        if (rc) return rc;
        chunks.push_back(std::move(b));
        ci = chunks.size() - 1;
        cur = 0;
    }
    *out = static_cast<char *>(chunks[ci].p) + cur;
    cur += bytes;
    return HSS_OK;
}

int Work::stage_bytes(const void *src, size_t bytes, void **dev) {
    int rc = dalloc_bytes(bytes, dev);
    if (rc || bytes == 0) return rc;
    size_t need = (bytes + 255) & ~(size_t)255;
    if (hused + need > hcap) {
        if (hpin) old_pins.push_back(hpin), old_sizes.push_back(hcap);   // copies in flight may still read it
        size_t want = std::max(need, std::max((size_t)(1u << 20), 2 * hcap));
        size_t got = 0;
        hpin = scratch_cache_take_pinned(need, want, got);
        hused = 0;
        hcap = got;
        if (!hpin) {
            hcap = 0;
            set_error("cudaMallocHost of the staging buffer failed");
            return HSS_ENOMEM;
        }
    }
    void *h = static_cast<char *>(hpin) + hused;
    std::memcpy(h, src, bytes);
    hused += need;
    cudaError_t e = cudaMemcpyAsync(*dev, h, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    return HSS_OK;
}

void Work::reset() {
    ci = 0;
    cur = 0;
    hused = 0;
    for (size_t k = 0; k < old_pins.size(); ++k) scratch_cache_give_pinned(old_pins[k], old_sizes[k]);
    old_pins.clear();
    old_sizes.clear();
}

}  // namespace hssnd

extern "C" {

const char *hss_last_error(void) { return hssnd::g_last_error.c_str(); }

long hss_alloc_count(void) { return hssnd::g_alloc_requests.load(std::memory_order_relaxed); }

void hss_nd_opts_default(hss_nd_opts *o) {
    if (!o) return;
    o->leaf_max = 64;
    o->scheme = HSS_SCHEME_BOX;
}

void hss_factor_opts_default(hss_factor_opts *o) {
    if (!o) return;
    o->tol = 1e-6;
    o->compress = 1;
    o->r0 = 32;
    o->dr = 32;
    o->rmax = 96;
    o->oversample = 10;
    o->precision = HSS_FP64;
    o->seed = 0;
    o->keep_schur = 0;
    o->tensor_cores = 0;
    o->r_init = nullptr;
    o->cap_policy = HSS_CAP_KEEP;
    o->autotune = 0;
    o->probe = 0;
    o->sample_bf16 = 0;
    o->merge = 0;
}

void fgmres_opts_default(fgmres_opts *o) {
    if (!o) return;
    o->restart = 30;
    o->rtol = 1e-8;
    o->maxit = 1000;
}

}  // extern "C"
