// hss_gemm_f32_static: the FP32 tile GEMM of hss_gemm_f32 with its launch
// records (one GEMM descriptor, the tile list, the tensor-core timeout flag)
// held in a fixed, file-scope device array instead of call workspace, so the
// call allocates no memory at all.
//
// Who needs it: a caller that runs where allocation is not allowed or not
// safe, e.g. inside a region that must not touch the allocator (a memory
// pool being trimmed or rebuilt, an allocator hook, a real-time loop with a
// fixed memory budget that has to leave the device heap untouched), or code
// that must not synchronize the device, which cudaFree does.
//
// Layout of the scratch (bytes from its 256-byte aligned start):
//   [0, 256)      GemmDesc<float> of the call
//   [256, 512)    int tensor-core timeout flag (zeroed by the setup kernel of
//                 every call before the GEMM reads it)
//   [512, ...)    GemmTile list, at most HSS_GEMM_STATIC_MAX_TILES entries
// Everything is written on the call's stream before the GEMM launch reads it,
// so nothing has to start at zero.  Two calls in flight at once (other
// streams, other host threads) share the array and race.
#include <mutex>

#include "hssnd.h"
#include "internal.h"
#include "prof.h"

namespace hssnd {

constexpr size_t STATIC_DESC_OFF = 0;
constexpr size_t STATIC_ERR_OFF = 256;
constexpr size_t STATIC_TILE_OFF = 512;
constexpr size_t STATIC_SCRATCH_BYTES = STATIC_TILE_OFF + sizeof(GemmTile) * HSS_GEMM_STATIC_MAX_TILES;
static_assert(sizeof(GemmDesc<float>) <= STATIC_ERR_OFF - STATIC_DESC_OFF, "descriptor slot too small");
static_assert(alignof(GemmTile) <= 16 && alignof(GemmDesc<float>) <= 256, "scratch alignment");

static __device__ __align__(256) unsigned char g_gemm_static_scratch[STATIC_SCRATCH_BYTES];

__global__ void k_gemm_static_setup(GemmDesc<float> d, int tm, int ntiles, GemmDesc<float> *dd, int *err,
                                    GemmTile *tiles);

constexpr int MAX_DEVICES = 64;
static std::mutex g_static_mu;
static unsigned char *g_static_addr[MAX_DEVICES];

// Device address of the scratch on the current device, looked up once per
// device.  The same first call also loads every kernel this entry point can
// launch (the SIMT and tensor-core GEMMs, the k = 0 kernel, the setup kernel)
// and sets the tensor-core kernel's shared-memory attribute, so after one
// call of any engine on a device no later call does module work.
static int static_scratch(unsigned char **out) {
    int dev = 0;
    HSS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("hss_gemm_f32_static: device ordinal beyond the supported 64");
        return HSS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gemm_static_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                     "cudaGetSymbolAddress(gemm static scratch)");
        int rc = gemm_f32_prepare();
        if (!rc) rc = gemm_tc_prepare();
        if (rc) return rc;
        cudaFuncAttributes fa;
        HSS_CUDA(cudaFuncGetAttributes(&fa, k_gemm_static_setup));
        g_static_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_addr[dev];
    return HSS_OK;
}

// Writes the descriptor, clears the timeout flag and lays out the full tile
// grid (tm x tn tiles, column of tiles after column) for the GEMM launch.
__global__ void k_gemm_static_setup(GemmDesc<float> d, int tm, int ntiles, GemmDesc<float> *dd, int *err,
                                    GemmTile *tiles) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *dd = d;
        *err = 0;
    }
    if (t < ntiles) tiles[t] = GemmTile{0, t % tm, t / tm};
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_gemm_f32_static(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C,
                                   int ldc, float alpha, float beta, int engine, void *stream) {
    if (m < 0 || n < 0 || k < 0 || !A || !B || !C || lda < std::max(1, m) || ldb < std::max(1, k) ||
        ldc < std::max(1, m) || engine < 0 || engine > 2) {
        set_error("hss_gemm_f32_static: invalid argument");
        return HSS_EINVAL;
    }
    if (m == 0 || n == 0) return HSS_OK;
    const int tile_m = engine == 0 ? GEMM_TM : GEMM_TC_TM, tile_n = engine == 0 ? GEMM_TN : GEMM_TC_TN;
    const long tm = cdiv(m, tile_m), tn = cdiv(n, tile_n);
    if (k > 0 && tm * tn > HSS_GEMM_STATIC_MAX_TILES) {   // (k = 0 needs no tile records)
        set_error("hss_gemm_f32_static: " + std::to_string(m) + " x " + std::to_string(n) + " needs " +
                  std::to_string(tm * tn) + " tiles of " + std::to_string(tile_m) + " x " + std::to_string(tile_n) +
                  ", more than the " + std::to_string(HSS_GEMM_STATIC_MAX_TILES) + " the fixed scratch holds");
        return HSS_EINVAL;
    }
    unsigned char *base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 0) {   // C = beta C: no product for any engine, no records needed
        if ((rc = gemm_f32_k0(C, ldc, m, n, alpha, beta, s))) return rc;
        HSS_CUDA(cudaStreamSynchronize(s));
        return HSS_OK;
    }
    GemmDesc<float> d{};
    d.A = A;
    d.B = B;
    d.C = C;
    d.lda = lda;
    d.ldb = ldb;
    d.ldc = ldc;
    d.m = m;
    d.n = n;
    d.k = k;
    d.alpha = alpha;
    d.beta = beta;
    auto *dd = reinterpret_cast<GemmDesc<float> *>(base + STATIC_DESC_OFF);
    auto *err = reinterpret_cast<int *>(base + STATIC_ERR_OFF);
    auto *dt = reinterpret_cast<GemmTile *>(base + STATIC_TILE_OFF);
    const int ntiles = (int)(tm * tn);
    {
        HSS_PROF("gemm_static_setup", s, 0.0);
        k_gemm_static_setup<<<cdiv(ntiles, 256), 256, 0, s>>>(d, (int)tm, ntiles, dd, err, dt);
        HSS_CHECK_LAUNCH("k_gemm_static_setup");
    }
    if (engine == 0)
        rc = gemm_batched<float>(dd, dt, ntiles, s, 2.0 * m * n * k);
    else
        rc = gemm_tc(dd, dt, ntiles, engine == 1 ? 1 : 0, err, s, 2.0 * m * n * k);
    if (rc) return rc;
    int herr = 0;
    HSS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("hss_gemm_f32_static: tensor-core wait timed out");
        return HSS_ETIMEOUT;
    }
    return HSS_OK;
}
