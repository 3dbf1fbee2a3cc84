// Batched tiled GEMM on a list of column-major problems (SIMT FMA, FP64 or
// FP32).  Serves the Gauss-Jordan trailing updates of the fronts (the Schur
// update S = F_bb - F_bi F_ii^-1 F_ib accumulates here), the randomized
// sampling products Y = S Omega, Z = S^t Psi with the +-1 test matrix
// generated in registers (never stored), and the leaf-local sample
// corrections of the HSS construction.
#include "internal.h"
#include "prof.h"

namespace hssnd {

constexpr int GK = 16;      // k-chunk
constexpr int GT = 256;     // threads per CTA (16 x 16, 4 x 4 outputs each)

template <class T>
__global__ void __launch_bounds__(GT) k_gemm(const GemmDesc<T> *__restrict__ descs, const GemmTile *__restrict__ tiles) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ T As[2][GK][GEMM_TM + 1];
    __shared__ T Bs[2][GK][GEMM_TN + 1];
    const GemmTile tl = tiles[blockIdx.x];
    const GemmDesc<T> d = descs[tl.desc];
    const int row0 = tl.tm * GEMM_TM, col0 = tl.tn * GEMM_TN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

    T ra[4], rb[4];
    auto load_regs = [&](int k0) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int idx = tid + GT * t;
            int i, kk;
            if (!d.transA) { i = idx & 63; kk = idx >> 6; }
            else { kk = idx & 15; i = idx >> 4; }
            int gi = row0 + i, gk = k0 + kk;
            T v = T(0);
            if (gi < d.m && gk < d.k) v = d.transA ? d.A[gk + (long)gi * d.lda] : d.A[gi + (long)gk * d.lda];
            ra[t] = v;
            int j;
            if (d.B && d.transB) { j = idx & 63; kk = idx >> 6; }
            else { kk = idx & 15; j = idx >> 4; }
            int gj = col0 + j;
            gk = k0 + kk;
            T w = T(0);
            if (gj < d.n && gk < d.k) {
                if (!d.B) w = (T)rademacher(d.seed, d.stream, d.front, d.brow0 + gk, gj);
                else w = d.transB ? d.B[gj + (long)gk * d.ldb] : d.B[gk + (long)gj * d.ldb];
            }
            rb[t] = w;
        }
    };
    auto store_regs = [&](int buf) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int idx = tid + GT * t;
            int i, kk, j;
            if (!d.transA) { i = idx & 63; kk = idx >> 6; }
            else { kk = idx & 15; i = idx >> 4; }
            As[buf][kk][i] = ra[t];
            if (d.B && d.transB) { j = idx & 63; kk = idx >> 6; }
            else { kk = idx & 15; j = idx >> 4; }
            Bs[buf][kk][j] = rb[t];
        }
    };
    int nk = (d.k + GK - 1) / GK;
    if (nk > 0) {
        load_regs(0);
        store_regs(0);
    }
    __syncthreads();
    for (int kc = 0; kc < nk; ++kc) {
        int buf = kc & 1;
        if (kc + 1 < nk) load_regs((kc + 1) * GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[buf][kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        if (kc + 1 < nk) store_regs(buf ^ 1);
        __syncthreads();
    }
    // the 16 C values this thread updates are loaded before any store (a store
    // could alias a later load: interleaved, they would run one at a time)
    T cv[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int gj = col0 + ty + 16 * b;
        const bool colok = gj < d.n && !(gj >= d.skip_lo && gj < d.skip_hi);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int gi = row0 + tx + 16 * a;
            const T beta = (gi >= d.zr_lo && gi < d.zr_hi) ? T(0) : d.beta;
            cv[a][b] = (colok && gi < d.m && beta != T(0)) ? d.C[gi + (long)gj * d.ldc] : T(0);
        }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int gj = col0 + ty + 16 * b;
        if (gj >= d.n || (gj >= d.skip_lo && gj < d.skip_hi)) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int gi = row0 + tx + 16 * a;
            if (gi >= d.m) continue;
            T beta = (gi >= d.zr_lo && gi < d.zr_hi) ? T(0) : d.beta;
            T v = d.alpha * acc[a][b];
            if (beta != T(0)) v = fma(beta, cv[a][b], v);
            d.C[gi + (long)gj * d.ldc] = v;
        }
    }
}

template <class T>
int gemm_batched(const GemmDesc<T> *d_desc, const GemmTile *d_tiles, int ntiles, cudaStream_t s, double flops) {
    if (ntiles <= 0) return HSS_OK;
    HSS_PROF(sizeof(T) == 8 ? "gemm_f64" : "gemm_f32", s, flops);
    HSS_CUDA(launch_pdl(k_gemm<T>, dim3(ntiles), dim3(GT), 0, s, d_desc, d_tiles));
    HSS_CHECK_LAUNCH("k_gemm");
    return HSS_OK;
}

template <class T>
void gemm_tiles_for(const GemmDesc<T> &d, int desc_index, std::vector<GemmTile> &tiles) {
    int tm = cdiv(d.m, GEMM_TM), tn = cdiv(d.n, GEMM_TN);
    for (int j = 0; j < tn; ++j) {
        // whole tile column inside the skipped column range: nothing to write
        int c0 = j * GEMM_TN, c1 = std::min(d.n, c0 + GEMM_TN);
        if (c0 >= d.skip_lo && c1 <= d.skip_hi) continue;
        for (int i = 0; i < tm; ++i) tiles.push_back({desc_index, i, j});
    }
}

// C = alpha * 0 + beta * C for a product with k = 0 (no descriptor, no
// allocation; the same arithmetic as k_gemm with an empty K loop).
__global__ void k_gemm_k0(float *__restrict__ C, int ldc, int m, int n, float alpha, float beta) {
    pdl_launch_next();
    pdl_wait_prev();
    const long tot = (long)m * n;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < tot; g += (long)gridDim.x * blockDim.x) {
        const int i = (int)(g % m), j = (int)(g / m);
        float *c = C + i + (long)j * ldc;
        float v = alpha * 0.f;
        if (beta != 0.f) v = fmaf(beta, *c, v);
        *c = v;
    }
}

int gemm_f32_k0(float *C, int ldc, int m, int n, float alpha, float beta, cudaStream_t s) {
    if (m <= 0 || n <= 0) return HSS_OK;
    HSS_PROF("gemm_f32", s, 0.0);
    HSS_CUDA(launch_pdl(k_gemm_k0, dim3((int)std::min<long>(cdiv((long)m * n, 256), 2 * 152 * 8)), dim3(256), 0, s, C, ldc, m, n, alpha, beta));
    HSS_CHECK_LAUNCH("k_gemm_k0");
    return HSS_OK;
}

// Loads the FP32 GEMM kernels' module (with lazy loading a kernel's module is
// loaded at its first launch or attribute query).
int gemm_f32_prepare() {
    cudaFuncAttributes fa;
    HSS_CUDA(cudaFuncGetAttributes(&fa, k_gemm<float>));
    HSS_CUDA(cudaFuncGetAttributes(&fa, k_gemm_k0));
    return HSS_OK;
}

template int gemm_batched<double>(const GemmDesc<double> *, const GemmTile *, int, cudaStream_t, double);
template int gemm_batched<float>(const GemmDesc<float> *, const GemmTile *, int, cudaStream_t, double);
template void gemm_tiles_for<double>(const GemmDesc<double> &, int, std::vector<GemmTile> &);
template void gemm_tiles_for<float>(const GemmDesc<float> &, int, std::vector<GemmTile> &);

}  // namespace hssnd
