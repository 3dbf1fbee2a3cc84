// Tensor-core GEMM for the FP32 (mixed) form: tcgen05.mma kind::tf32 on sm_103a,
// accumulator in tensor memory (TMEM), FP32 accuracy by the three-product
// split A B ~= Ah Bh + Ah Bl + Al Bh (hi = tf32(x), lo = tf32(x - hi)).
//
// One CTA (128 threads) per 128 x 128 tile of C; K in chunks of 32.  Operands
// are staged by the CTA's threads into shared memory in the canonical K-major,
// non-swizzled UMMA layout: core matrices of 8 rows x 16 bytes, rows 16 bytes
// apart, core matrices 128 bytes apart along K (LBO) and 8-row groups 1024
// bytes apart (SBO).  One thread issues the MMAs and commits them to an
// mbarrier; all threads wait (bounded), then read the accumulator with
// tcgen05.ld and apply C = alpha * acc + beta * C with the same row/column
// masks as the SIMT kernel (gemm.cu).  Same descriptor list and semantics as
// k_gemm<float>, including the +-1 test-matrix operand generated on the fly.
#include <cstdint>

#include "internal.h"
#include "prof.h"

namespace hssnd {

namespace {

constexpr int TC_M = GEMM_TC_TM;
constexpr int TC_N = GEMM_TC_TN;
constexpr int TC_K = 32;            // K per staged chunk
constexpr int TC_NT = 128;          // threads per CTA
constexpr uint32_t TC_LBO = 128;    // bytes between core matrices along K
constexpr uint32_t TC_SBO = 1024;   // bytes between 8-row groups (TC_K / 4 core matrices x 128 B)
constexpr int TC_TILE_BYTES = TC_M * TC_K * 4;   // one operand tile (16 KB)
constexpr long TC_SPIN_LIMIT = 1L << 26;         // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of element (row, k) of a K-major tile in the canonical layout
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
    return (uint32_t)((row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture; no swizzle, base offset 0
    return d;
}

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

}  // namespace

// One 128 x 128 tile of one problem per CTA.  Tiles are in units of 128.
// spin_limit bounds every mbarrier wait; issue = 0 stages the operands but
// issues no MMA and no commit, so the first wait runs out (the self-test of
// the timeout path: nothing is left in flight when the kernel returns).
__global__ void __launch_bounds__(TC_NT) k_gemm_tc(const GemmDesc<float> *__restrict__ descs,
                                                   const GemmTile *__restrict__ tiles, int split,
                                                   int *__restrict__ err, long spin_limit, int issue) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    // 1024-byte aligned operand tiles: Ahi, Bhi, Alo, Blo
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sAh = base, *sBh = base + TC_TILE_BYTES;
    unsigned char *sAl = base + 2 * TC_TILE_BYTES, *sBl = base + 3 * TC_TILE_BYTES;

    const GemmTile tl = tiles[blockIdx.x];
    const GemmDesc<float> d = descs[tl.desc];
    const int row0 = tl.tm * TC_M, col0 = tl.tn * TC_N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_tf32(TC_M, TC_N);

    uint32_t phase = 0;
    bool timed_out = false;
    const int nk = (d.k + TC_K - 1) / TC_K;
    for (int kc = 0; kc < nk && !timed_out; ++kc) {
        const int k0 = kc * TC_K;
        // stage A (128 rows x 32 k) and B^t (128 cols x 32 k), hi and lo parts
        for (int idx = tid; idx < TC_M * TC_K; idx += TC_NT) {
            int i, kk;
            if (!d.transA) { i = idx & (TC_M - 1); kk = idx >> 7; }
            else { kk = idx & (TC_K - 1); i = idx >> 5; }
            const int gi = row0 + i, gk = k0 + kk;
            float a = 0.f;
            if (gi < d.m && gk < d.k) a = d.transA ? d.A[gk + (long)gi * d.lda] : d.A[gi + (long)gk * d.lda];
            const uint32_t hi = to_tf32(a);
            const uint32_t lo = to_tf32(a - __uint_as_float(hi));
            const uint32_t off = kmaj_off(i, kk);
            *reinterpret_cast<uint32_t *>(sAh + off) = hi;
            *reinterpret_cast<uint32_t *>(sAl + off) = lo;
        }
        for (int idx = tid; idx < TC_N * TC_K; idx += TC_NT) {
            int j, kk;
            if (d.B && d.transB) { j = idx & (TC_N - 1); kk = idx >> 7; }
            else { kk = idx & (TC_K - 1); j = idx >> 5; }
            const int gj = col0 + j, gk = k0 + kk;
            float b = 0.f;
            if (gj < d.n && gk < d.k) {
                if (!d.B) b = (float)rademacher(d.seed, d.stream, d.front, d.brow0 + gk, gj);
                else b = d.transB ? d.B[gj + (long)gk * d.ldb] : d.B[gk + (long)gj * d.ldb];
            }
            const uint32_t hi = to_tf32(b);
            const uint32_t lo = to_tf32(b - __uint_as_float(hi));
            const uint32_t off = kmaj_off(j, kk);
            *reinterpret_cast<uint32_t *>(sBh + off) = hi;
            *reinterpret_cast<uint32_t *>(sBl + off) = lo;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && issue) {
            tc_fence_after();
            const uint32_t aH = smem_u32(sAh), bH = smem_u32(sBh), aL = smem_u32(sAl), bL = smem_u32(sBl);
#pragma unroll
            for (int s = 0; s < TC_K / 8; ++s) {   // 8 tf32 per MMA = two core matrices along K
                const uint32_t so = (uint32_t)s * 2 * TC_LBO;
                const int acc0 = (kc > 0 || s > 0) ? 1 : 0;
                mma_tf32(tmem, smem_desc(aH + so), smem_desc(bH + so), idesc, acc0);
                if (split) {
                    mma_tf32(tmem, smem_desc(aH + so), smem_desc(bL + so), idesc, 1);
                    mma_tf32(tmem, smem_desc(aL + so), smem_desc(bH + so), idesc, 1);
                }
            }
            mma_commit(&bar);
        }
        // every thread waits for the MMAs (they read this chunk's shared memory);
        // the wait is bounded and the timeout decision is made block-uniform
        long spins = 0;
        bool mine = false;
        while (!mbar_try_wait(&bar, phase)) {
            if (++spins > spin_limit) {
                mine = true;
                break;
            }
        }
        phase ^= 1u;
        tc_fence_after();
        timed_out = __syncthreads_or(mine) != 0;
    }
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
        // let the MMAs in flight finish (bounded) before the accumulator is freed
        long spins = 0;
        while (issue && !mbar_try_wait(&bar, phase ^ 1u) && ++spins < spin_limit) {
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 16 columns at a time
        const int gi = row0 + warp * 32 + lane;
        const bool rowok = gi < d.m;
        const float beta_row = (gi >= d.zr_lo && gi < d.zr_hi) ? 0.f : d.beta;
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            float v[16];
            if (nk > 0) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {   // k = 0: no MMA wrote the accumulator, A B is zero
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
            if (!rowok) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int gj = col0 + c0 + q;
                if (gj >= d.n || (gj >= d.skip_lo && gj < d.skip_hi)) continue;
                float *c = d.C + gi + (long)gj * d.ldc;
                float val = d.alpha * v[q];
                if (beta_row != 0.f) val = fmaf(beta_row, *c, val);
                *c = val;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

constexpr size_t TC_SMEM = 4 * TC_TILE_BYTES + 1024;

// The dynamic shared-memory attribute of k_gemm_tc, set once per device
// (thread-safe; the attribute is per device context).  Setting it also loads
// the kernel's module, so a call made early takes that work out of later ones.
int gemm_tc_prepare() {
    HSS_SMEM(k_gemm_tc, TC_SMEM);
    return HSS_OK;
}

static int launch_tc(const GemmDesc<float> *d_desc, const GemmTile *d_tiles, int ntiles, int split, int *err,
                     cudaStream_t s, double flops, long spin_limit, int issue) {
    if (ntiles <= 0) return HSS_OK;
    int rc = gemm_tc_prepare();
    if (rc) return rc;
    HSS_PROF("gemm_tc", s, flops);
    HSS_CUDA(launch_pdl(k_gemm_tc, dim3(ntiles), dim3(TC_NT), TC_SMEM, s, d_desc, d_tiles, split, err, spin_limit, issue));
    HSS_CHECK_LAUNCH("k_gemm_tc");
    return HSS_OK;
}

int gemm_tc(const GemmDesc<float> *d_desc, const GemmTile *d_tiles, int ntiles, int split, int *err, cudaStream_t s,
            double flops) {
    return launch_tc(d_desc, d_tiles, ntiles, split, err, s, flops, TC_SPIN_LIMIT, 1);
}

void gemm_tc_tiles_for(const GemmDesc<float> &d, int desc_index, std::vector<GemmTile> &tiles) {
    int tm = cdiv(d.m, TC_M), tn = cdiv(d.n, TC_N);
    for (int j = 0; j < tn; ++j) {
        int c0 = j * TC_N, c1 = std::min(d.n, c0 + TC_N);
        if (c0 >= d.skip_lo && c1 <= d.skip_hi) continue;
        for (int i = 0; i < tm; ++i) tiles.push_back({desc_index, i, j});
    }
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_gemm_f32(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                            float alpha, float beta, int engine, void *stream) {
    if (m < 0 || n < 0 || k < 0 || !A || !B || !C || lda < std::max(1, m) || ldb < std::max(1, k) ||
        ldc < std::max(1, m) || engine < 0 || engine > 3) {
        set_error("hss_gemm_f32: invalid argument");
        return HSS_EINVAL;
    }
    if (m == 0 || n == 0) return HSS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 0) {   // C = beta C: no product for any engine to run
        int rc0 = gemm_f32_k0(C, ldc, m, n, alpha, beta, s);
        if (rc0) return rc0;
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
    if (engine == 3 && !gemm_tma_eligible(d)) engine = 1;   // operands TMA cannot address
    std::vector<GemmTile> tiles;
    if (engine == 0)
        gemm_tiles_for(d, 0, tiles);
    else
        gemm_tc_tiles_for(d, 0, tiles);
    Work W(s);
    GemmDesc<float> *dd;
    GemmTile *dt;
    int *err;
    std::vector<GemmDesc<float>> dv{d};
    int rc;
    if ((rc = W.up(dv, &dd)) || (rc = W.up(tiles, &dt)) || (rc = W.dalloc(1, &err))) return rc;
    HSS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (engine == 0) {
        rc = gemm_batched<float>(dd, dt, (int)tiles.size(), s, 2.0 * m * n * k);
    } else if (engine == 3) {
        TmaGemmDesc *td;
        if ((rc = gemm_tma_descs(dv, std::vector<char>{1}, W, &td))) return rc;
        rc = gemm_tma(td, dt, (int)tiles.size(), err, s, 2.0 * m * n * k);
    } else {
        rc = gemm_tc(dd, dt, (int)tiles.size(), engine == 1 ? 1 : 0, err, s, 2.0 * m * n * k);
    }
    if (rc) return rc;
    int herr = 0;
    HSS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("hss_gemm_f32: tensor-core wait timed out");
        return HSS_ETIMEOUT;
    }
    return HSS_OK;
}

// Test hook of the bounded tensor-core wait: one CTA of k_gemm_tc on a
// 128 x 128 x 32 problem that issues no MMA, so its mbarrier never completes
// and the wait gives up after spin_limit polls.
extern "C" int hss_tc_timeout_selftest(long spin_limit, void *stream) {
    if (spin_limit < 1 || spin_limit > TC_SPIN_LIMIT) {
        set_error("hss_tc_timeout_selftest: spin_limit out of range");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Work W(s);
    float *buf;
    GemmDesc<float> *dd;
    GemmTile *dt;
    int *err;
    int rc;
    if ((rc = W.dalloc((size_t)3 * TC_M * TC_N, &buf)) || (rc = W.dalloc(1, &err))) return rc;
    HSS_CUDA(cudaMemsetAsync(buf, 0, sizeof(float) * 3 * TC_M * TC_N, s));
    HSS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    GemmDesc<float> d{};
    d.A = buf;
    d.B = buf + TC_M * TC_N;
    d.C = buf + 2 * TC_M * TC_N;
    d.lda = d.ldc = TC_M;
    d.ldb = TC_K;
    d.m = TC_M;
    d.n = TC_N;
    d.k = TC_K;
    d.alpha = 1.f;
    std::vector<GemmDesc<float>> dv{d};
    std::vector<GemmTile> tv{{0, 0, 0}};
    if ((rc = W.up(dv, &dd)) || (rc = W.up(tv, &dt))) return rc;
    if ((rc = launch_tc(dd, dt, 1, 0, err, s, 0.0, spin_limit, 0))) return rc;
    int herr = 0;
    HSS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("hss_tc_timeout_selftest: the bounded tensor-core wait expired");
        return HSS_ETIMEOUT;
    }
    return HSS_OK;
}
