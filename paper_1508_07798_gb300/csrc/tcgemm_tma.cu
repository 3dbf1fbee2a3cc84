// Tensor-core GEMM fed by TMA: tcgen05.mma kind::tf32 whose operand tiles
// are brought into shared memory by cp.async.bulk.tensor (one tensor map per
// operand and problem), K in chunks of 16, so the copies of later chunks
// overlap the work on the current one.
//
// Same problem list, tiles (128 x 128 of C) and semantics as k_gemm<float> /
// k_gemm_tc (gemm.cu, tcgemm.cu): C = alpha op(A) op(B) + beta C with the
// row/column masks, B = NULL meaning the +-1 test matrix of the counter hash.
//
// Per chunk:
//   1. TMA copies the raw FP32 tiles (no swizzle) into a 2-deep ring: an
//      operand whose rows run along M/N in memory (A not transposed, B
//      transposed) arrives as four boxes of 32 rows x 16 K, each K a 128-byte
//      line; an operand with K contiguous as one box of 16 K x 128 rows,
//      64-byte lines.
//   2. The threads split every value x into hi = tf32(x), lo = tf32(x - hi)
//      and write both into the canonical K-major, non-swizzled tcgen05 layout
//      (core matrices of 8 rows x 16 bytes, 128 B apart along K, 8-row groups
//      512 B apart), double-buffered; the +-1 operand is generated there.
//      The raw slot is free again as soon as the threads have read it.
//   3. One thread issues hiA hiB + hiA loB + loA hiB (hiA B + loA B for the
//      exact +-1 B) and commits to the buffer's mbarrier.
// The MMAs of a chunk overlap the conversion of the next and the copies of
// the two after it.  Every mbarrier wait is bounded (2 s of the global timer)
// and sets the error flag when it gives up.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "prof.h"

namespace hssnd {

namespace {

constexpr int TM = 128, TN = 128, TK = 16;   // output tile, K per chunk
constexpr int NT = 256;                      // 8 warps: two per TMEM lane quarter
constexpr int OPB = TM * TK * 4;             // bytes of one operand tile of a chunk (8 KB)
constexpr int RAW_BYTES = 2 * OPB;           // raw A, raw B of one ring slot
constexpr int CONV_BYTES = 4 * OPB;          // A hi, A lo, B hi, B lo of one buffer
constexpr size_t SMEM = 2 * (size_t)RAW_BYTES + 2 * (size_t)CONV_BYTES + 1024;
constexpr uint32_t LBO = 128, SBO = 512;     // canonical K-major layout of a 16-K tile
constexpr unsigned long long WAIT_NS = 2000000000ull;   // a bounded wait gives up after 2 s
constexpr long SPIN_CAP = 1L << 30;                       // and after this many polls in any case

enum { OP_MN = 0, OP_K = 1, OP_GEN = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// descriptor of K-step ks (8 tf32 = two core matrices along K) of a converted tile
__device__ __forceinline__ uint64_t kdesc(uint32_t base, int ks) {
    const uint32_t addr = base + (uint32_t)ks * 2u * LBO;
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// byte offset of element (row, k) in the canonical K-major tile
__device__ __forceinline__ uint32_t koff(int row, int k) {
    return (uint32_t)((row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4);
}

// byte offset of element (row, k) in a raw TMA tile
__device__ __forceinline__ uint32_t raw_off(int mode, int row, int k) {
    return mode == OP_MN ? (uint32_t)((row >> 5) * 2048 + k * 128 + (row & 31) * 4) : (uint32_t)(row * 64 + k * 4);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
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

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: false when it gave up (2 s of the global timer)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = gtime();
    for (long spins = 1; spins < SPIN_CAP; ++spins) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((spins & 255) == 0 && gtime() - t0 > WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
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

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// ---- BF16 sampling (kind::f16): A as three BF16 terms, the exact +-1 B in BF16.
// Canonical K-major layout of a 16-K BF16 tile: core matrices of 8 rows x 16
// bytes (8 values along K), 128 B apart along K, 8-row groups 256 B apart.
constexpr uint32_t LBO16 = 128, SBO16 = 256;
constexpr int OPB16 = TM * TK * 2;   // bytes of one BF16 tile of a chunk (4 KB)

__device__ __forceinline__ uint32_t koff16(int row, int k) {
    return (uint32_t)((row >> 3) * SBO16 + (k >> 3) * LBO16 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t kdesc16(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((LBO16 >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((SBO16 >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// round to nearest BF16 (bit pattern), and back
__device__ __forceinline__ unsigned short to_bf16(float x) {
    unsigned short r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float from_bf16(unsigned short b) { return __uint_as_float((uint32_t)b << 16); }

}  // namespace

// One problem of the TMA engine: the tensor maps of its operands and its
// GemmDesc (aligned like CUtensorMap, 128 bytes; TMA needs at least 64).
struct alignas(128) TmaGemmDesc {
    CUtensorMap ta;
    CUtensorMap tb;
    GemmDesc<float> d;
    int amode, bmode;
};

namespace {

// TMA copies of chunk kc into a raw ring slot (thread 0)
__device__ __forceinline__ void issue_chunk(const TmaGemmDesc *td, int amode, int bmode, int row0, int col0, int kc,
                                            unsigned char *slot, uint64_t *full) {
    const int k0 = kc * TK;
    const uint32_t a = smem_u32(slot), b = smem_u32(slot + OPB);
    mbar_expect_tx(full, (uint32_t)(OPB + (bmode == OP_GEN ? 0 : OPB)));
    if (amode == OP_MN) {
#pragma unroll
        for (int q = 0; q < TM / 32; ++q) tma_load_2d(a + q * 2048u, &td->ta, row0 + 32 * q, k0, full);
    } else {
        tma_load_2d(a, &td->ta, k0, row0, full);
    }
    if (bmode == OP_MN) {
#pragma unroll
        for (int q = 0; q < TN / 32; ++q) tma_load_2d(b + q * 2048u, &td->tb, col0 + 32 * q, k0, full);
    } else if (bmode == OP_K) {
        tma_load_2d(b, &td->tb, k0, col0, full);
    }
}

// raw tile (layout `mode`) -> hi and lo tiles in the canonical K-major layout;
// each thread handles 4 consecutive K of one row
__device__ __forceinline__ void convert_tile(const unsigned char *raw, int mode, unsigned char *hi, unsigned char *lo) {
    for (int q = threadIdx.x; q < TM * TK / 4; q += NT) {
        const int row = q & (TM - 1), k4 = (q >> 7) * 4;
        float4 h, l;
        float *hs = reinterpret_cast<float *>(&h), *ls = reinterpret_cast<float *>(&l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float x = *reinterpret_cast<const float *>(raw + raw_off(mode, row, k4 + u));
            const uint32_t hb = to_tf32(x);
            hs[u] = __uint_as_float(hb);
            ls[u] = __uint_as_float(to_tf32(x - __uint_as_float(hb)));
        }
        const uint32_t o = koff(row, k4);
        *reinterpret_cast<float4 *>(hi + o) = h;
        *reinterpret_cast<float4 *>(lo + o) = l;
    }
}

// raw FP32 tile (layout `mode`) -> three BF16 terms x ~ t0 + t1 + t2 (each
// the BF16 rounding of what the previous terms left), canonical K-major BF16
// layout; each thread handles 8 consecutive K of one row
__device__ __forceinline__ void convert_tile_bf16(const unsigned char *raw, int mode, unsigned char *t0,
                                                  unsigned char *t1, unsigned char *t2) {
    for (int q = threadIdx.x; q < TM * TK / 8; q += NT) {
        const int row = q & (TM - 1), k8 = (q >> 7) * 8;
        unsigned short h[8], m[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float x = *reinterpret_cast<const float *>(raw + raw_off(mode, row, k8 + u));
            h[u] = to_bf16(x);
            const float r1 = x - from_bf16(h[u]);
            m[u] = to_bf16(r1);
            l[u] = to_bf16(r1 - from_bf16(m[u]));
        }
        const uint32_t o = koff16(row, k8);
        *reinterpret_cast<uint4 *>(t0 + o) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(t1 + o) = *reinterpret_cast<const uint4 *>(m);
        *reinterpret_cast<uint4 *>(t2 + o) = *reinterpret_cast<const uint4 *>(l);
    }
}

}  // namespace

template <bool BF16>
__global__ void __launch_bounds__(NT, 2) k_gemm_tma(const TmaGemmDesc *__restrict__ descs,
                                                  const GemmTile *__restrict__ tiles, int *__restrict__ err) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t full[2];     // raw slot landed (TMA transaction count)
    __shared__ __align__(8) uint64_t mdone[2];    // MMAs reading converted buffer b finished
    __shared__ uint32_t tmem_base;
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    unsigned char *rawb = base;                       // 2 raw slots
    unsigned char *conv = base + 2 * RAW_BYTES;       // 2 converted buffers

    const GemmTile tl = tiles[blockIdx.x];
    const TmaGemmDesc *td = descs + tl.desc;
    const GemmDesc<float> d = td->d;
    const int amode = td->amode, bmode = td->bmode;
    const int row0 = tl.tm * TM, col0 = tl.tn * TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = (d.k + TK - 1) / TK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&mdone[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = 0; q < 2 && q < nk; ++q) issue_chunk(td, amode, bmode, row0, col0, q, rawb + q * RAW_BYTES, &full[q]);
    }
    // the epilogue reads C: start bringing this tile's C into L2 now (thread t:
    // column col0 + t, the rows of the tile that exist, in 128-byte lines)
    {
        const int pc = col0 + (tid & (TN - 1)), half = tid >> 7;   // column, half of the tile's rows
        if (d.beta != 0.f && pc < d.n && !(pc >= d.skip_lo && pc < d.skip_hi)) {
            const float *cc = d.C + row0 + (long)pc * d.ldc;
            const int rows = min(TM, d.m - row0);
            for (int r = half * (TM / 2); r < min(rows, (half + 1) * (TM / 2)); r += 32)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cc + r));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = BF16 ? idesc_bf16() : idesc_tf32();

    bool failed = false;
    int issued = nk < 2 ? nk : 2;   // chunks whose copies were issued (thread 0's view)
    int kc_stop = nk;               // first chunk not consumed
    int committed = 0;              // MMA commits per converted buffer (thread 0)
    for (int kc = 0; kc < nk; ++kc) {
        const int q = kc & 1;
        const uint32_t ph = (uint32_t)(kc >> 1) & 1u;
        unsigned char *raw = rawb + q * RAW_BYTES;
        unsigned char *cb = conv + q * CONV_BYTES;
        // the raw slot has landed, and the MMAs of chunk kc - 2 no longer read buffer q
        bool bad = !mbar_wait(&full[q], ph);
        if (kc >= 2) bad = bad || !mbar_wait(&mdone[q], (uint32_t)((kc - 2) >> 1) & 1u);
        if (__syncthreads_or(bad)) {
            failed = true;
            kc_stop = kc;
            break;
        }
        if constexpr (BF16) {   // A in three BF16 terms, the +-1 B in BF16 (the host routes only generated B here)
            convert_tile_bf16(raw, amode, cb, cb + OPB16, cb + 2 * OPB16);
            unsigned char *bt = cb + 3 * OPB16;
            const int k0 = kc * TK;
            for (int idx = tid; idx < TN * TK; idx += NT) {
                const int kk = idx & (TK - 1), j = idx >> 4;
                const int gj = col0 + j, gk = k0 + kk;
                unsigned short v = 0;
                if (gj < d.n && gk < d.k)
                    v = rademacher(d.seed, d.stream, d.front, d.brow0 + gk, gj) > 0 ? (unsigned short)0x3F80
                                                                                   : (unsigned short)0xBF80;
                *reinterpret_cast<unsigned short *>(bt + koff16(j, kk)) = v;
            }
        } else {
        convert_tile(raw, amode, cb, cb + OPB);
        if (bmode == OP_GEN) {
            unsigned char *bt = cb + 2 * OPB;
            const int k0 = kc * TK;
            for (int idx = tid; idx < TN * TK; idx += NT) {
                const int kk = idx & (TK - 1), j = idx >> 4;
                const int gj = col0 + j, gk = k0 + kk;
                float v = 0.f;
                if (gj < d.n && gk < d.k) v = (float)rademacher(d.seed, d.stream, d.front, d.brow0 + gk, gj);
                *reinterpret_cast<float *>(bt + koff(j, kk)) = v;
            }
        } else {
            convert_tile(raw + OPB, bmode, cb + 2 * OPB, cb + 3 * OPB);
        }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();   // every thread is done with the raw slot and the buffer is written
        if (tid == 0) {
            tc_fence_after();
            if (issued < nk) {   // the raw slot is free: copy chunk kc + 2 into it
                issue_chunk(td, amode, bmode, row0, col0, issued, raw, &full[q]);
                ++issued;
            }
            if constexpr (BF16) {   // one K = 16 MMA per term
                const uint32_t a0 = smem_u32(cb), b0 = a0 + 3 * OPB16;
                const uint64_t bd = kdesc16(b0);
                mma_bf16(tmem, kdesc16(a0), bd, idesc, kc > 0 ? 1 : 0);
                mma_bf16(tmem, kdesc16(a0 + OPB16), bd, idesc, 1);
                mma_bf16(tmem, kdesc16(a0 + 2 * OPB16), bd, idesc, 1);
            } else {
            const uint32_t aH = smem_u32(cb), aL = aH + OPB, bH = aH + 2 * OPB, bL = aH + 3 * OPB;
#pragma unroll
            for (int ks = 0; ks < TK / 8; ++ks) {
                const int acc0 = (kc > 0 || ks > 0) ? 1 : 0;
                mma_tf32(tmem, kdesc(aH, ks), kdesc(bH, ks), idesc, acc0);
                if (bmode != OP_GEN) mma_tf32(tmem, kdesc(aH, ks), kdesc(bL, ks), idesc, 1);
                mma_tf32(tmem, kdesc(aL, ks), kdesc(bH, ks), idesc, 1);
            }
            }
            mma_commit(&mdone[q]);
            ++committed;
        }
    }
    // every MMA issued has finished: the last commit of each buffer covers it
    bool ok = true;
    if (!failed) {
        for (int q = 0; q < 2 && q < nk; ++q) {
            const int last = (nk - 1 - q) - ((nk - 1 - q) & 1) + q;   // last chunk of buffer q
            ok = ok && mbar_wait(&mdone[q], (uint32_t)(last >> 1) & 1u);
        }
    }
    failed = __syncthreads_or(failed || !ok) != 0;
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            // copies issued for chunks not consumed land before the block leaves (bounded)
            for (int c = kc_stop; c < issued; ++c) mbar_wait(&full[c & 1], (uint32_t)(c >> 1) & 1u);
            // and the MMAs committed so far finish
            if (committed > 0) {
                for (int q = 0; q < 2; ++q) {
                    const int cnt = q == 0 ? (committed + 1) / 2 : committed / 2;   // commits on buffer q
                    if (cnt > 0) mbar_wait(&mdone[q], (uint32_t)(cnt - 1) & 1u);
                }
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quarter:
        // rows) and the columns of half w / 4, 32 at a time; the 32 C values of
        // a row are loaded together before any store (a store could alias a
        // later load, so loads interleaved with stores would run one round trip
        // at a time)
        const int quarter = warp & 3, chalf = warp >> 2;
        const int gi = row0 + quarter * 32 + lane;
        const bool rowok = gi < d.m;
        const float beta_row = (gi >= d.zr_lo && gi < d.zr_hi) ? 0.f : d.beta;
        constexpr int EC = 16;
        for (int c0 = chalf * (TN / 2); c0 < (chalf + 1) * (TN / 2); c0 += EC) {
            float v[EC], cv[EC];
#pragma unroll
            for (int u = 0; u < EC; ++u) {
                const int gj = col0 + c0 + u;
                const bool ok = rowok && gj < d.n && !(gj >= d.skip_lo && gj < d.skip_hi) && beta_row != 0.f;
                cv[u] = ok ? d.C[gi + (long)gj * d.ldc] : 0.f;
            }
            if (nk > 0) {
#pragma unroll
                for (int q = 0; q < EC; q += 16)
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c0 + q), v + q);
            } else {
#pragma unroll
                for (int u = 0; u < EC; ++u) v[u] = 0.f;
            }
            if (!rowok) continue;
#pragma unroll
            for (int u = 0; u < EC; ++u) {
                const int gj = col0 + c0 + u;
                if (gj >= d.n || (gj >= d.skip_lo && gj < d.skip_hi)) continue;
                float val = d.alpha * v[u];
                if (beta_row != 0.f) val = fmaf(beta_row, cv[u], val);
                d.C[gi + (long)gj * d.ldc] = val;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool aligned16(const void *p, long ld) {
    return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld > 0 && (ld * 4) % 16 == 0;
}

// 2D FP32 map: inner x outer elements, row stride ld elements
bool encode(CUtensorMap *map, const float *ptr, long inner, long outer, long ld, int box0, int box1) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tma_eligible(const GemmDesc<float> &d) {
    if (d.m < 1 || d.n < 1 || d.k < 1 || !encode_fn()) return false;
    if (!aligned16(d.A, d.lda)) return false;
    if (d.B && !aligned16(d.B, d.ldb)) return false;
    return true;
}

int gemm_tma_prepare() {
    HSS_SMEM(k_gemm_tma<false>, SMEM);
    HSS_SMEM(k_gemm_tma<true>, SMEM);
    return HSS_OK;
}

// Tensor maps of every problem flagged in `use` (the others are left zero and
// must not appear in the tile list), uploaded through W.
int gemm_tma_descs(const std::vector<GemmDesc<float>> &descs, const std::vector<char> &use, Work &W,
                   TmaGemmDesc **out) {
    std::vector<TmaGemmDesc> td(descs.size());
    std::memset(static_cast<void *>(td.data()), 0, sizeof(TmaGemmDesc) * td.size());
    for (size_t i = 0; i < descs.size(); ++i) {
        if (!use[i]) continue;
        const GemmDesc<float> &d = descs[i];
        TmaGemmDesc &t = td[i];
        t.d = d;
        bool ok;
        if (!d.transA) {   // A(i, kk) at i + lda kk: M contiguous
            t.amode = OP_MN;
            ok = encode(&t.ta, d.A, d.m, d.k, d.lda, 32, TK);
        } else {           // A(i, kk) at kk + lda i: K contiguous
            t.amode = OP_K;
            ok = encode(&t.ta, d.A, d.k, d.m, d.lda, TK, TM);
        }
        if (!d.B) {
            t.bmode = OP_GEN;
        } else if (!d.transB) {   // B(kk, j) at kk + ldb j: K contiguous
            t.bmode = OP_K;
            ok = ok && encode(&t.tb, d.B, d.k, d.n, d.ldb, TK, TN);
        } else {                  // B(kk, j) at j + ldb kk: N contiguous
            t.bmode = OP_MN;
            ok = ok && encode(&t.tb, d.B, d.n, d.k, d.ldb, 32, TK);
        }
        if (!ok) {
            set_error("tensor-core GEMM: tensor map encoding failed");
            return HSS_ECUDA;
        }
    }
    // the scratch hands out 256-byte aligned pieces: every map stays 128-byte aligned
    return W.up(td, out);
}

int gemm_tma(const TmaGemmDesc *d_descs, const GemmTile *d_tiles, int ntiles, int *err, cudaStream_t s,
             double flops, const char *prof_class, bool bf16) {
    if (ntiles <= 0) return HSS_OK;
    int rc = gemm_tma_prepare();
    if (rc) return rc;
    HSS_PROF(prof_class, s, flops);
    if (bf16)
        HSS_CUDA(launch_pdl(k_gemm_tma<true>, dim3(ntiles), dim3(NT), SMEM, s, d_descs, d_tiles, err));
    else
        HSS_CUDA(launch_pdl(k_gemm_tma<false>, dim3(ntiles), dim3(NT), SMEM, s, d_descs, d_tiles, err));
    HSS_CHECK_LAUNCH("k_gemm_tma");
    return HSS_OK;
}

}  // namespace hssnd
