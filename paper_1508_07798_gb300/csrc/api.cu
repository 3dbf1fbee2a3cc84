// Error state, option defaults and small shared host utilities of libhssnd.
#include <cstdio>
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
}

void fgmres_opts_default(fgmres_opts *o) {
    if (!o) return;
    o->restart = 30;
    o->rtol = 1e-8;
    o->maxit = 1000;
}

}  // extern "C"
