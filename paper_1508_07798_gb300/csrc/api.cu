// Error state, option defaults and small shared host utilities of libhssnd.
#include <cstdio>
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace hssnd {

static thread_local std::string g_last_error;

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

Work::~Work() {
    cudaStreamSynchronize(s);
    chunks.clear();
    if (hpin) cudaFreeHost(hpin);
    for (void *p : old_pins) cudaFreeHost(p);
}

int Work::dalloc_bytes(size_t bytes, void **out) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (chunks.empty() || cur + bytes > chunks.back().bytes) {
        size_t want = std::max(bytes, std::max((size_t)(16u << 20), chunks.empty() ? 0 : 2 * chunks.back().bytes));
        DevBuf b;
        int rc = b.alloc(want);
        if (rc) return rc;
        chunks.push_back(std::move(b));
        cur = 0;
    }
    *out = static_cast<char *>(chunks.back().p) + cur;
    cur += bytes;
    return HSS_OK;
}

int Work::stage_bytes(const void *src, size_t bytes, void **dev) {
    int rc = dalloc_bytes(bytes, dev);
    if (rc || bytes == 0) return rc;
    size_t need = (bytes + 255) & ~(size_t)255;
    if (hused + need > hcap) {
        if (hpin) old_pins.push_back(hpin);   // copies in flight may still read it
        hcap = std::max(need, std::max((size_t)(1u << 20), 2 * hcap));
        hused = 0;
        if (cudaMallocHost(&hpin, hcap) != cudaSuccess) {
            hpin = nullptr;
            hcap = 0;
            return cuda_fail(cudaGetLastError(), "cudaMallocHost");
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
    if (chunks.size() > 1) {
        size_t total = 0;
        for (auto &c : chunks) total += c.bytes;
        chunks.clear();
        DevBuf b;
        if (b.alloc(total) == HSS_OK) chunks.push_back(std::move(b));
    }
    cur = 0;
    hused = 0;
    for (void *p : old_pins) cudaFreeHost(p);
    old_pins.clear();
}

}  // namespace hssnd

extern "C" {

const char *hss_last_error(void) { return hssnd::g_last_error.c_str(); }

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
}

void fgmres_opts_default(fgmres_opts *o) {
    if (!o) return;
    o->restart = 30;
    o->rtol = 1e-8;
    o->maxit = 1000;
}

}  // extern "C"
