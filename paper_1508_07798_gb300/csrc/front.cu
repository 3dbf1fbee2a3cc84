// Front assembly and front elimination.
//
// A front sigma holds the dofs [I ; B] (I = I^sigma at a leaf, I^sigma above;
// Sec. 4.1).  Its matrix F is assembled from the stored blocks of A (leaf:
// all of A(front, front); parent: the cross couplings A(B^mu, B^nu), eq. (32))
// while the children's HSS approximants are written in by the compression
// step.  Elimination is a blocked Gauss-Jordan sweep over the I pivots with
// partial (row) pivoting inside I.  It turns F in place into
//
//     [ F_ii^-1 P^t          F_ii^-1 F_ib            ]      (W = M(B,I)^t)
//     [ -F_bi F_ii^-1 P^t    F_bb - F_bi F_ii^-1 F_ib ]      (-L(B,I), S)
//
// i.e. the inverse of the D block and both Gauss transforms of Sec. 4.1 plus
// the Schur complement of eq. (32).  P is the pivot row permutation; the
// apply undoes it by gathering x_I through a permuted index list.
#include <cfloat>
#include <mutex>
#include <type_traits>

#include <cooperative_groups.h>

#include "internal.h"
#include "front.h"
#include "prof.h"

namespace hssnd {

// ---------------------------------------------------------------- assembly
// One warp per front element: copy every stored block (e, f) with f in the
// same front (leaf fronts) or in the other child (parent fronts) into F.
template <class T>
__global__ void k_scatter_A(const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                            const double *__restrict__ val, int bs, const StageElem *__restrict__ se, int nse,
                            const int *__restrict__ elem_slot, const FrontDev *__restrict__ fr, T *__restrict__ arena) {
    pdl_launch_next();
    pdl_wait_prev();
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= nse) return;
    const StageElem me = se[w];
    const FrontDev F = fr[me.front];
    T *M = arena + F.foff;
    int bs2 = bs * bs;
    for (int t = row_ptr[me.elem]; t < row_ptr[me.elem + 1]; ++t) {
        int f = col_idx[t];
        int sf = elem_slot[f];
        if (sf < 0) continue;
        const StageElem other = se[sf];
        if (other.front != me.front) continue;
        if (!F.leaf && other.side == me.side) continue;
        const double *blk = val + (long)t * bs2;
        for (int q = lane; q < bs2; q += 32) {
            int r = q / bs, c = q % bs;
            M[(me.fpos + r) + (long)F.n * (other.fpos + c)] = (T)blk[q];
        }
    }
}

__global__ void k_set_slots(const StageElem *__restrict__ se, int nse, int *__restrict__ elem_slot, int value_is_index) {
    pdl_launch_next();
    pdl_wait_prev();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nse) elem_slot[se[i].elem] = value_is_index ? i : -1;
}

// ---------------------------------------------------------------- GJ panel
// Argmax over non-negative magnitudes by their IEEE bit patterns (monotonic
// for v >= 0; -1 = no candidate), so no floating-point compare is spent on the
// reduction (FP64 compares run on GB300's narrow FP64 pipe).
template <class T> struct ArgMax {
    long long v;
    int i;
};
__device__ __forceinline__ long long mag_key(float a) { return (long long)(__float_as_int(a) & 0x7fffffff); }
__device__ __forceinline__ long long mag_key(double a) { return __double_as_longlong(a) & 0x7fffffffffffffffLL; }

// Block-wide argmax (largest |v|, ties to the lowest index) with one barrier:
// every thread reduces the per-warp results itself.  The caller guarantees a
// barrier between two calls (so nobody still reads sh when it is rewritten).
// Warp argmax of (key, position): largest key, lowest position on ties; every
// lane gets the result.
template <class T> __device__ __forceinline__ ArgMax<T> warp_argmax(ArgMax<T> x) {
    if constexpr (std::is_same<T, float>::value) {
        // FP32 magnitude keys fit in 31 bits; +1 maps "no candidate" (-1) to 0.
        // Two warp reductions: the largest key, then the lowest position holding it.
        const unsigned k = (unsigned)(x.v + 1);
        const unsigned m = __reduce_max_sync(0xffffffffu, k);
        const int pos = __reduce_min_sync(0xffffffffu, k == m ? x.i : 0x7fffffff);
        return ArgMax<T>{(long long)m - 1, pos};
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            const long long v2 = __shfl_xor_sync(0xffffffffu, x.v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, x.i, o);
            if (v2 > x.v || (v2 == x.v && i2 < x.i)) {
                x.v = v2;
                x.i = i2;
            }
        }
        return x;
    }
}

template <class T> __device__ ArgMax<T> block_argmax(ArgMax<T> x, ArgMax<T> *sh) {
    x = warp_argmax(x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    // every warp reduces the per-warp results (at most 32) in parallel
    ArgMax<T> y{-1LL, 0x7fffffff};
    if (lane < nw) y = sh[lane];
    return warp_argmax(y);
}

// One CTA per front with an active panel [k0, k0+kb) of its I columns.
// 1. Gauss-Jordan on the tall panel rows [k0, ni) x panel columns, with row
//    pivoting inside [k0+j, ni) (in shared memory when it fits);
// 2. the pivot row swaps applied to the columns outside the panel, and to the
//    running row permutation rperm (position -> original I row);
// 3. Aold = pivot rows, all columns (input of the trailing update);
// 4. rows outside [k0, ni): F(i, P) = -F(i, P) X with X = F(P,P)^-1;
// 5. last panel of a front: the apply's gather list iperm[j] = I[rperm[j]]
//    (the sweep leaves F_ii^-1 P^t, so F_ii^-1 x = (F_ii^-1 P^t)(P x)).
template <class T>
__global__ void __launch_bounds__(PANEL_NT) k_gj_panel(const PanelJob *__restrict__ jobs, const FrontDev *__restrict__ fr,
                                                    T *__restrict__ arena, T *__restrict__ xws,
                                                    int *__restrict__ mws, int *__restrict__ piv,
                                                    int *__restrict__ rperm, const int *__restrict__ ilist,
                                                    int *__restrict__ iperm, int *__restrict__ status) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ ArgMax<T> red[PANEL_NT / 32];
    __shared__ T rowj[PANEL_KB_MAX];
    __shared__ int swp[PANEL_KB_MAX];
    const PanelJob J = jobs[blockIdx.x];
    const FrontDev F = fr[J.front];
    T *M = arena + F.foff;
    const long ld = F.n;
    const int k0 = J.k0, kb = J.kb, ni = F.ni, n = F.n;
    const int hT = ni - k0;
    T *P;
    long ldp;
    int *rp;   // rperm[k0 .. ni) in shared memory
    if (J.smem) {
        P = reinterpret_cast<T *>(smraw);
        ldp = hT;
        rp = reinterpret_cast<int *>(smraw + sizeof(T) * (size_t)hT * kb);
        const int tot = hT * kb;
        for (int q0 = threadIdx.x; q0 < tot; q0 += PANEL_NT * 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int q = q0 + u * PANEL_NT;
                v[u] = q < tot ? M[(k0 + q % hT) + ld * (k0 + q / hT)] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int q = q0 + u * PANEL_NT;
                if (q < tot) P[(q % hT) + ldp * (q / hT)] = v[u];
            }
        }
    } else {
        P = M + k0 + ld * k0;
        ldp = ld;
        rp = reinterpret_cast<int *>(smraw);
    }
    int *rglob = rperm + F.ioff;
    for (int i = threadIdx.x; i < hT; i += PANEL_NT) rp[i] = k0 == 0 ? i : rglob[k0 + i];
    __syncthreads();
    int *pv = piv + F.ioff;
    // candidates of the first pivot column (rows below the pivot limit)
    const int hP = min(hT, J.rlim - k0);
    ArgMax<T> loc{-1LL, 0x7fffffff};
    for (int i = threadIdx.x; i < hP; i += PANEL_NT) {
        long long a = mag_key(P[i]);
        if (a > loc.v) {
            loc.v = a;
            loc.i = i;
        }
    }
    for (int j = 0; j < kb; ++j) {
        // 1. pivot: largest |P(i, j)| over i >= j, ties to the lowest row
        ArgMax<T> best = block_argmax(loc, red);
        int p = best.i;
        if (best.v <= 0) {
            if (threadIdx.x == 0) atomicExch(&status[J.front], 1);
            p = j;
        }
        // 2. swap rows j and p inside the panel; the pivot row goes to rowj
        for (int c = threadIdx.x; c < kb; c += PANEL_NT) {
            T pj = P[p + ldp * c];
            if (p != j) P[p + ldp * c] = P[j + ldp * c];
            P[j + ldp * c] = pj;
            rowj[c] = pj;
        }
        if (threadIdx.x == 0) {
            pv[k0 + j] = k0 + p;
            swp[j] = p;
            int t = rp[j];
            rp[j] = rp[p];
            rp[p] = t;
        }
        __syncthreads();
        // 3. eliminate column j from every other row, finish row j, and gather
        //    the candidates of column j+1 (rows > j) on the way
        const T dinv = rowj[j] != T(0) ? T(1) / rowj[j] : T(0);
        loc = ArgMax<T>{-1LL, 0x7fffffff};
        for (int i = threadIdx.x; i < hT; i += PANEL_NT) {
            if (i == j) {
                for (int c = 0; c < kb; ++c) P[j + ldp * c] = (c == j) ? dinv : rowj[c] * dinv;
                continue;
            }
            const T a = P[i + ldp * j];
            if (a != T(0)) {
                const T ad = a * dinv;
#pragma unroll 8
                for (int c = 0; c < kb; ++c) P[i + ldp * c] -= ad * rowj[c];
                P[i + ldp * j] = -ad;
            }
            if (i > j && j + 1 < kb && i < hP) {
                long long v2 = mag_key(P[i + ldp * (j + 1)]);
                if (v2 > loc.v) {
                    loc.v = v2;
                    loc.i = i;
                }
            }
        }
        // the barrier inside the next block_argmax orders these writes
    }
    __syncthreads();
    // X = inverse of the pivot block, for the rows outside the panel
    T *Xg = xws + J.xoff;
    for (int q = threadIdx.x; q < kb * kb; q += PANEL_NT) {
        int i = q % kb, c = q / kb;
        Xg[q] = P[i + ldp * c];
    }
    if (J.smem) {
        // write the panel back, eight loads in flight per thread
        const int tot = hT * kb;
        for (int q0 = threadIdx.x; q0 < tot; q0 += PANEL_NT * 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int q = q0 + u * PANEL_NT;
                v[u] = q < tot ? P[(q % hT) + ldp * (q / hT)] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int q = q0 + u * PANEL_NT;
                if (q < tot) M[(k0 + q % hT) + ld * (k0 + q / hT)] = v[u];
            }
        }
    }
    for (int i = threadIdx.x; i < hT; i += PANEL_NT) rglob[k0 + i] = rp[i];
    // the panel's swaps compose to a permutation that moves at most 2 kb rows:
    // moves[0] = count, moves[1..64] = destinations, moves[65..128] = sources.
    // q (position -> source position) lives in shared memory for the touched
    // positions only: slot t < kb is position t, slot kb + j is position swp[j].
    __shared__ int qpos[2 * PANEL_KB_MAX], qsrc[2 * PANEL_KB_MAX];
    __shared__ int nmv;
    if (threadIdx.x < 2 * kb) {
        int x = threadIdx.x < kb ? threadIdx.x : swp[threadIdx.x - kb];
        qpos[threadIdx.x] = x;
        qsrc[threadIdx.x] = x;
    }
    if (threadIdx.x == 0) nmv = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        // slot of position x: x < kb -> x; otherwise the first kb + j with swp[j] == x
        auto slot = [&](int x) {
            if (x < kb) return x;
            for (int j = 0; j < kb; ++j)
                if (swp[j] == x) return kb + j;
            return -1;
        };
        for (int j = 0; j < kb; ++j) {
            int pj = swp[j];
            if (pj == j) continue;
            int a = j, b = slot(pj);
            int t = qsrc[a];
            qsrc[a] = qsrc[b];
            qsrc[b] = t;
        }
    }
    __syncthreads();
    int *mv = mws + J.moff;
    if (threadIdx.x < 2 * kb) {
        int t = threadIdx.x;
        int x = qpos[t];
        // keep the first slot of each position only
        bool first = t < kb || x >= kb;
        if (t >= kb)
            for (int j = 0; j < t - kb; ++j)
                if (swp[j] == x) first = false;
        if (first && qsrc[t] != x) {
            int m = atomicAdd(&nmv, 1);
            mv[1 + m] = x;
            mv[1 + 2 * PANEL_KB_MAX + m] = qsrc[t];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) mv[0] = nmv;
    // last panel: gather list of the apply
    if (k0 + kb == ni) {
        __syncthreads();
        for (int j = threadIdx.x; j < ni; j += PANEL_NT) {
            int r = j < k0 ? rglob[j] : rp[j - k0];
            iperm[F.iperm_off + j] = ilist[F.iset_off + r];
        }
    }
}

// One warp's pivot candidate at one step of the register panel: the largest
// |value| of the active column among its rows (ties to the lowest position),
// that row's position and panel row, and the row's KB register values.
template <class T, int KB> struct __align__(16) PanelCand {
    T v[KB];
    long long key;   // -1: the warp has no candidate
    int pos, row;
};

template <class T, int KB> __device__ __forceinline__ void put_row(T *dst, const T (&src)[KB]) {
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int c = 0; c < KB; c += 4)
            *reinterpret_cast<float4 *>(dst + c) = make_float4(src[c], src[c + 1], src[c + 2], src[c + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < KB; c += 2) *reinterpret_cast<double2 *>(dst + c) = make_double2(src[c], src[c + 1]);
    }
}

// 16 bytes of a shared-memory row, loaded where the code asks for them (the
// pivot row is re-read per owned row instead of being held in registers).
template <class T> __device__ __forceinline__ void get_vec(const T *src, T *dst) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(src);
    if constexpr (std::is_same<T, float>::value)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(dst[0]), "=f"(dst[1]), "=f"(dst[2]), "=f"(dst[3])
                     : "r"(a));
    else
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(dst[0]), "=d"(dst[1]) : "r"(a));
}

// Register-resident panel: thread t owns panel rows t, t + NT, ... (R rows of
// KB values each) for the whole panel.  Rows are not moved while pivoting:
// each thread keeps its rows' current positions in registers and replays the
// interchanges of partial pivoting exactly (the search runs over rows not yet
// pivoted and below the pivot limit, ties to the lowest position); every row
// is written once, to its final position.
// One barrier per pivot step: every warp publishes its best candidate row to
// a double-buffered shared slot, and after the barrier every thread reduces
// the NT/32 slots and reads the pivot row from the winning one.  The pivot
// loop runs in unrolled groups of U steps, so the active column sits in a
// register fixed at compile time; the registers rotate left by U once per
// group (after G groups register c holds column (G U + c) mod KB).
template <class T, int KB, int R, int NT>
__global__ void __launch_bounds__(NT) k_gj_panel_reg(const PanelJob *__restrict__ jobs,
                                                        const FrontDev *__restrict__ fr, T *__restrict__ arena,
                                                        T *__restrict__ xws, int *__restrict__ mws,
                                                        int *__restrict__ piv, int *__restrict__ rperm,
                                                        const int *__restrict__ ilist, int *__restrict__ iperm,
                                                        int *__restrict__ status) {
    pdl_launch_next();
    pdl_wait_prev();
    constexpr int NW = NT / 32;
    // steps per rotation group: fewer where the rows fill more of the register budget
    constexpr int DREGS = R * KB * (int)sizeof(T) / 4;
    constexpr int U = (NT > 256 || DREGS > 64) ? 1 : DREGS <= 48 ? 4 : 2;
    constexpr int V = 16 / (int)sizeof(T);   // values per 16-byte shared load
    // row positions in registers for up to two rows per thread, else in shared memory
    constexpr bool POS_REG = R <= 2;
    static_assert(KB % U == 0 && KB > U && U <= 4, "panel width");
    __shared__ PanelCand<T, KB> cand[2][NW];
    __shared__ int pos_s[POS_REG ? 1 : R * NT];
    __shared__ int swp[KB];   // pivot position of each step
    __shared__ int nmv, zero_piv;
    const PanelJob J = jobs[blockIdx.x];
    const FrontDev F = fr[J.front];
    T *M = arena + F.foff;
    const long ld = F.n;
    const int k0 = J.k0, kb = J.kb, ni = F.ni;
    const int hT = ni - k0;
    const int hP = min(hT, J.rlim - k0);   // pivot candidates: positions below hP
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *rglob = rperm + F.ioff;
    // position of owned row q; a pivoted row keeps its position j as
    // j - PIV_DONE (negative); rows past hT keep positions >= hP
    constexpr int PIV_DONE = 1 << 30;
    int pos_r[POS_REG ? R : 1];
    auto getpos = [&](int q) -> int {
        if constexpr (POS_REG)
            return pos_r[q];
        else
            return pos_s[threadIdx.x + NT * q];
    };
    auto setpos = [&](int q, int v) {
        if constexpr (POS_REG)
            pos_r[q] = v;
        else
            pos_s[threadIdx.x + NT * q] = v;
    };
    T reg[R][KB];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = threadIdx.x + NT * q;
        setpos(q, i);
#pragma unroll
        for (int c = 0; c < KB; ++c) reg[q][c] = (i < hT && c < kb) ? M[(k0 + i) + ld * (k0 + c)] : T(0);
    }
    if (threadIdx.x == 0) {
        nmv = 0;
        zero_piv = 0;
    }
    // candidates of the first column
    ArgMax<T> loc{-1LL, 0x7fffffff};
    int lq = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int ps = getpos(q);
        if (ps >= 0 && ps < hP) {
            const long long v = mag_key(reg[q][0]);
            if (v > loc.v || (v == loc.v && ps < loc.i)) {
                loc.v = v;
                loc.i = ps;
                lq = q;
            }
        }
    }
#pragma unroll 1
    for (int g = 0; g < kb; g += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = g + u;
            if (j < kb) {   // uniform over the block
                // 1. this warp's candidate to its slot
                PanelCand<T, KB> *slot = cand[j & 1];
                const ArgMax<T> wb = warp_argmax(loc);
                const unsigned own = __ballot_sync(0xffffffffu, loc.v >= 0 && loc.v == wb.v && loc.i == wb.i);
                if (own == 0u) {
                    if (lane == 0) slot[w].key = -1LL;
                } else if (lane == __ffs(own) - 1) {
                    slot[w].key = wb.v;
                    slot[w].pos = wb.i;
                    slot[w].row = threadIdx.x + NT * lq;
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (q == lq) put_row<T, KB>(slot[w].v, reg[q]);
                }
                __syncthreads();
                // 2. the pivot: best slot (largest key, lowest position)
                ArgMax<T> y{-1LL, 0x7fffffff};
                if (lane < NW) {
                    const long long k = slot[lane].key;
                    if (k >= 0) y = ArgMax<T>{k, slot[lane].pos};
                }
                const ArgMax<T> best = warp_argmax(y);
                const unsigned wm = __ballot_sync(0xffffffffu, lane < NW && y.v >= 0 && y.v == best.v && y.i == best.i);
                // (position j always holds a candidate, so wm != 0; an empty wm would
                // leave every row in place and is reported as a zero pivot)
                const int ws = wm ? __ffs(wm) - 1 : 0;
                const T *prow = slot[ws].v;
                const int p = wm ? best.i : j, x = wm ? slot[ws].row : -1;
                if (threadIdx.x == 0) {
                    swp[j] = p;
                    if (best.v <= 0) zero_piv = 1;
                }
                // 3. Gauss-Jordan step, row by row (every row, then the pivot row overwritten)
                const T pj = prow[u];
                const T dinv = pj != T(0) ? T(1) / pj : T(0);
                loc = ArgMax<T>{-1LL, 0x7fffffff};
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const bool isx = threadIdx.x + NT * q == x;
                    const T ad = reg[q][u] * dinv;
#pragma unroll
                    for (int c0 = 0; c0 < KB; c0 += V) {
                        T rv[V];
                        get_vec<T>(prow + c0, rv);
#pragma unroll
                        for (int e = 0; e < V; ++e)
                            if (c0 + e != u) reg[q][c0 + e] -= ad * rv[e];
                    }
                    reg[q][u] = -ad;
                    if (__builtin_expect(isx, 0)) {   // the pivot row: one thread of the block
#pragma unroll
                        for (int c0 = 0; c0 < KB; c0 += V) {
                            T rv[V];
                            get_vec<T>(prow + c0, rv);
#pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (c0 + e != u) reg[q][c0 + e] = rv[e] * dinv;
                        }
                        reg[q][u] = dinv;
                    }
                    int ps = getpos(q);
                    if (isx)
                        setpos(q, j - PIV_DONE);
                    else if (ps == j)
                        setpos(q, ps = p);   // the row at position j trades places with the pivot
                    // 4. candidates of the next column (register u + 1 of this group)
                    if (!isx && ps >= 0 && ps < hP) {
                        const long long v = mag_key(reg[q][u + 1]);
                        if (v > loc.v || (v == loc.v && ps < loc.i)) {
                            loc.v = v;
                            loc.i = ps;
                            lq = q;
                        }
                    }
                }
            }
        }
        // rotate left by U
#pragma unroll
        for (int q = 0; q < R; ++q) {
            T t[U];
#pragma unroll
            for (int c = 0; c < U; ++c) t[c] = reg[q][c];
#pragma unroll
            for (int c = 0; c + U < KB; ++c) reg[q][c] = reg[q][c + U];
#pragma unroll
            for (int c = 0; c < U; ++c) reg[q][KB - U + c] = t[c];
        }
    }
    // original I rows of the owned rows, read before any thread rewrites rperm
    int orow[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = threadIdx.x + NT * q;
        orow[q] = i < hT ? (k0 == 0 ? i : rglob[k0 + i]) : 0;
    }
    __syncthreads();
    // every row to its final position; the pivot block also to X
    const int S = U * ((kb + U - 1) / U);
    T *Xg = xws + J.xoff;
    int *mv = mws + J.moff;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = threadIdx.x + NT * q;
        if (i >= hT) continue;
        const int ps = getpos(q);
        const int r = ps < 0 ? ps + PIV_DONE : ps;
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            const int col = (S + c) % KB;
            if (col < kb) {
                M[(k0 + r) + ld * (k0 + col)] = reg[q][c];
                if (r < kb) Xg[r + kb * col] = reg[q][c];
            }
        }
        rglob[k0 + r] = orow[q];
        if (r != i) {   // the other columns move the same way (k_gj_post)
            int m = atomicAdd(&nmv, 1);
            mv[1 + m] = r;
            mv[1 + 2 * PANEL_KB_MAX + m] = i;
        }
    }
    if (threadIdx.x < kb) piv[F.ioff + k0 + threadIdx.x] = k0 + swp[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        mv[0] = nmv;
        if (zero_piv) atomicExch(&status[J.front], 1);
    }
    if (k0 + kb == ni)
        for (int j = threadIdx.x; j < ni; j += NT) iperm[F.iperm_off + j] = ilist[F.iset_off + rglob[j]];
}

// Cluster-resident panel for tall panels (more rows than one CTA's registers
// hold): a cluster of CL CTAs shares one panel, CTA c thread t owning rows
// q (CL NT) + c NT + t, q < R, in registers.  Per pivot: every CTA reduces its
// rows' candidates, the CL candidates are exchanged through distributed
// shared memory (largest magnitude, lowest position on ties: the pivot of the
// single-CTA kernel), the owner publishes the pivot row and every CTA reads
// it from the owner's shared memory; the Gauss-Jordan step then runs in
// registers as in k_gj_panel_reg.  The row <-> position bookkeeping (pos,
// posinv, rp) is replicated in every CTA (the same swaps, applied by each),
// so CTA 0 alone writes the global bookkeeping (pivots, rperm, move list,
// gather list) and every CTA writes its own rows to their final positions.
namespace cg = cooperative_groups;

template <class T, int KB, int R, int NT, int CL>
__global__ void __launch_bounds__(NT) k_gj_panel_cl(const PanelJob *__restrict__ jobs,
                                                       const FrontDev *__restrict__ fr, T *__restrict__ arena,
                                                       T *__restrict__ xws, int *__restrict__ mws,
                                                       int *__restrict__ piv, int *__restrict__ rperm,
                                                       const int *__restrict__ ilist, int *__restrict__ iperm,
                                                       int *__restrict__ status) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ ArgMax<T> red[NT / 32];
    __shared__ ArgMax<T> cand;        // this CTA's best candidate of the current step
    __shared__ ArgMax<T> gbest;       // the cluster's pivot of the current step
    __shared__ T rowx[KB];            // the pivot row, when this CTA owns it
    __shared__ T rowj[KB];            // the pivot row, local copy
    __shared__ int nmv;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const PanelJob J = jobs[blockIdx.x / CL];
    const FrontDev F = fr[J.front];
    T *M = arena + F.foff;
    const long ld = F.n;
    const int k0 = J.k0, kb = J.kb, ni = F.ni;
    const int hT = ni - k0;
    constexpr int STRIDE = CL * NT;
    int *pos = reinterpret_cast<int *>(smraw);   // hT, replicated
    int *posinv = pos + hT;                       // hT
    int *rp = posinv + hT;                        // hT
    int *rglob = rperm + F.ioff;
    T reg[R][KB];
    bool done[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = q * STRIDE + crank * NT + threadIdx.x;
        done[q] = false;
#pragma unroll
        for (int c = 0; c < KB; ++c) reg[q][c] = (i < hT && c < kb) ? M[(k0 + i) + ld * (k0 + c)] : T(0);
    }
    for (int i = threadIdx.x; i < hT; i += NT) {
        pos[i] = i;
        posinv[i] = i;
        rp[i] = k0 == 0 ? i : rglob[k0 + i];
    }
    if (threadIdx.x == 0) nmv = 0;
    __syncthreads();
    int *pv = piv + F.ioff;
    const int hP = min(hT, J.rlim - k0);   // pivot candidates: positions below the limit
    ArgMax<T> loc{-1LL, 0x7fffffff};
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = q * STRIDE + crank * NT + threadIdx.x;
        if (i < hP) {
            const long long v = mag_key(reg[q][0]);
            if (v > loc.v || (v == loc.v && i < loc.i)) {
                loc.v = v;
                loc.i = i;
            }
        }
    }
#pragma unroll 1
    for (int j = 0; j < kb; ++j) {
        // 1. this CTA's best, then the cluster's (warp 0 reads the CL candidates)
        const ArgMax<T> mine = block_argmax(loc, red);
        if (threadIdx.x == 0) cand = mine;
        cluster.sync();
        if (threadIdx.x < 32) {
            ArgMax<T> c{-1LL, 0x7fffffff};
            if ((int)threadIdx.x < CL) c = *cluster.map_shared_rank(&cand, (unsigned)threadIdx.x);
            c = warp_argmax(c);
            if (threadIdx.x == 0) gbest = c;
        }
        __syncthreads();
        const ArgMax<T> best = gbest;
        int p = best.i;
        if (best.v <= 0) {
            if (threadIdx.x == 0 && crank == 0) atomicExch(&status[J.front], 1);
            p = j;
        }
        const int x = posinv[p];   // row of the pivot
        const int y = posinv[j];   // row at position j: trades places with the pivot
        const int owner = (x % STRIDE) / NT;
        if (owner == crank) {
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (q * STRIDE + crank * NT + (int)threadIdx.x == x) {
#pragma unroll
                    for (int c = 0; c < KB; ++c) rowx[c] = reg[q][c];
                }
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (q * STRIDE + crank * NT + (int)threadIdx.x == x) done[q] = true;
        cluster.sync();   // rowx of the owner is complete; every CTA has read cand and posinv
        if (threadIdx.x < KB) rowj[threadIdx.x] = cluster.map_shared_rank(rowx, (unsigned)owner)[threadIdx.x];
        if (threadIdx.x == 0) {
            posinv[j] = x;
            posinv[p] = y;
            pos[x] = j;
            pos[y] = p;
            const int t = rp[j];
            rp[j] = rp[p];
            rp[p] = t;
            if (crank == 0) pv[k0 + j] = k0 + p;
        }
        __syncthreads();
        // 2. Gauss-Jordan step in registers, then rotate; candidates of the next column
        const T dinv = rowj[0] != T(0) ? T(1) / rowj[0] : T(0);
        loc = ArgMax<T>{-1LL, 0x7fffffff};
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = q * STRIDE + crank * NT + threadIdx.x;
            if (i >= hT) continue;
            T head;
            if (i == x) {
#pragma unroll
                for (int c = 1; c < KB; ++c) reg[q][c] = rowj[c] * dinv;
                head = dinv;
            } else {
                const T ad = reg[q][0] * dinv;
#pragma unroll
                for (int c = 1; c < KB; ++c) reg[q][c] -= ad * rowj[c];
                head = -ad;
            }
#pragma unroll
            for (int c = 0; c + 1 < KB; ++c) reg[q][c] = reg[q][c + 1];
            reg[q][KB - 1] = head;
            if (!done[q]) {
                const long long v = mag_key(reg[q][0]);
                const int ps = (i == y) ? p : pos[i];
                if (ps < hP && (v > loc.v || (v == loc.v && ps < loc.i))) {
                    loc.v = v;
                    loc.i = ps;
                }
            }
        }
    }
    __syncthreads();
    // 3. every row to its final position; the pivot block also to X
    T *Xg = xws + J.xoff;
    int *mv = mws + J.moff;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = q * STRIDE + crank * NT + threadIdx.x;
        if (i >= hT) continue;
        const int r = pos[i];
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            const int col = (kb + c) % KB;
            if (col < kb) {
                M[(k0 + r) + ld * (k0 + col)] = reg[q][c];
                if (r < kb) Xg[r + kb * col] = reg[q][c];
            }
        }
    }
    if (crank == 0) {
        // the move list (rows whose position changed) and the bookkeeping, from the replica
        for (int i = threadIdx.x; i < hT; i += NT) {
            const int r = pos[i];
            if (r != i) {
                const int m = atomicAdd(&nmv, 1);
                mv[1 + m] = r;
                mv[1 + 2 * PANEL_KB_MAX + m] = i;
            }
            rglob[k0 + i] = rp[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) mv[0] = nmv;
        if (k0 + kb == ni)
            for (int jj = threadIdx.x; jj < ni; jj += NT) {
                const int r = jj < k0 ? rglob[jj] : rp[jj - k0];
                iperm[F.iperm_off + jj] = ilist[F.iset_off + r];
            }
    }
    cluster.sync();   // no CTA leaves while a peer may still read its shared memory
}

// Work that follows a panel, spread over many CTAs:
//   type 0 (32 columns outside the panel): apply the panel's row moves, then
//          copy the (moved) pivot rows into Aold, the B operand of the update;
//   type 1 (64 rows outside [k0, ni)): F(i, P) <- -F(i, P) X.
template <class T>
__global__ void __launch_bounds__(256) k_gj_post(const PanelTile *__restrict__ tiles, const PanelJob *__restrict__ jobs,
                                             const FrontDev *__restrict__ fr, T *__restrict__ arena,
                                             T *__restrict__ aold_ws, const T *__restrict__ xws,
                                             const int *__restrict__ mws) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ T Xs[PANEL_KB_MAX * PANEL_KB_MAX];
    __shared__ T old[64][PANEL_KB_MAX + 1];
    const PanelTile tl = tiles[blockIdx.x];
    const PanelJob J = jobs[tl.job];
    const FrontDev F = fr[J.front];
    T *M = arena + F.foff;
    const long ld = F.n;
    const int k0 = J.k0, kb = J.kb, n = F.n, hT = F.ni - k0;
    if (tl.type == 0) {
        const int *mv = mws + J.moff;
        const int nm = mv[0];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        T *Ao = aold_ws + J.aoff;
        for (int cc = wid; cc < 32; cc += 8) {
            const int c = tl.start + cc;
            if (c >= n || c < tl.c_lo || c >= tl.c_hi || (c >= k0 && c < k0 + kb)) continue;
            T *col = M + ld * c + k0;
            if (nm > 0) {
                T v0 = lane < nm ? col[mv[1 + 2 * PANEL_KB_MAX + lane]] : T(0);
                T v1 = lane + 32 < nm ? col[mv[1 + 2 * PANEL_KB_MAX + lane + 32]] : T(0);
                __syncwarp();
                if (lane < nm) col[mv[1 + lane]] = v0;
                if (lane + 32 < nm) col[mv[1 + lane + 32]] = v1;
                __syncwarp();
            }
            if (lane < kb) Ao[lane + (long)kb * c] = col[lane];
        }
        return;
    }
    // type 1
    const T *Xg = xws + J.xoff;
    for (int q = threadIdx.x; q < kb * kb; q += 256) Xs[q] = Xg[q];
    const int nout = n - hT;
    const int rr = threadIdx.x & 63, cg4 = threadIdx.x >> 6;   // 64 rows x 4 column groups
    const int r = tl.start + rr;
    const int i = r < k0 ? r : r + hT;
    if (r < nout)
        for (int s2 = cg4; s2 < kb; s2 += 4) old[rr][s2] = M[i + ld * (k0 + s2)];
    __syncthreads();
    if (r < nout)
        for (int c = cg4; c < kb; c += 4) {
            T acc = T(0);
            for (int s2 = 0; s2 < kb; ++s2) acc = fma(old[rr][s2], Xs[s2 + kb * c], acc);
            M[i + ld * (k0 + c)] = -acc;
        }
}

// End of a block of panels, for the columns outside the block (32 per tile):
// replay the row moves of the block's panels in order, then copy the block's
// pivot rows [k0, k0 + width) into Aold, the B operand of the block's update.
template <class T>
__global__ void __launch_bounds__(256) k_gj_block_post(const BlockTile *__restrict__ tiles,
                                                   const BlockJob *__restrict__ bjobs,
                                                   const PanelJob *__restrict__ jobs,
                                                   const FrontDev *__restrict__ fr, T *__restrict__ arena,
                                                   T *__restrict__ aold_ws, const int *__restrict__ mws) {
    pdl_launch_next();
    pdl_wait_prev();
    const BlockTile tl = tiles[blockIdx.x];
    const BlockJob B = bjobs[tl.bjob];
    const FrontDev F = fr[B.front];
    T *M = arena + F.foff;
    const long ld = F.n;
    const int n = F.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *Ao = aold_ws + B.aoff;
    for (int cc = wid; cc < 32; cc += 8) {
        const int c = tl.start + cc;
        if (c >= n || (c >= B.k0 && c < B.k0 + B.width)) continue;
        for (int q = 0; q < B.np; ++q) {
            const PanelJob J = jobs[B.job[q]];
            const int *mv = mws + J.moff;
            const int nm = mv[0];
            if (nm == 0) continue;
            T *col = M + ld * c + J.k0;
            T v0 = lane < nm ? col[mv[1 + 2 * PANEL_KB_MAX + lane]] : T(0);
            T v1 = lane + 32 < nm ? col[mv[1 + 2 * PANEL_KB_MAX + lane + 32]] : T(0);
            __syncwarp();
            if (lane < nm) col[mv[1 + lane]] = v0;
            if (lane + 32 < nm) col[mv[1 + lane + 32]] = v1;
            __syncwarp();
        }
        const T *colk = M + ld * c + B.k0;
        for (int i = lane; i < B.width; i += 32) Ao[i + (long)B.width * c] = colk[i];
    }
}

// ---------------------------------------------------------------- launchers
template <class T>
int launch_scatter_A(const hss_bsr *A, const StageElem *se, int nse, int *elem_slot, const FrontDev *fr, T *arena,
                     cudaStream_t s) {
    if (nse == 0) return HSS_OK;
    { HSS_PROF("set_slots", s); HSS_CUDA(launch_pdl(k_set_slots, dim3(cdiv(nse, 256)), dim3(256), 0, s, se, nse, elem_slot, 1)); }
    { HSS_PROF("scatter_A", s);
    HSS_CUDA(launch_pdl(k_scatter_A<T>, dim3(cdiv((long)nse * 32, 256)), dim3(256), 0, s, A->row_ptr, A->col_idx, A->val, A->bs, se, nse,
                                                             elem_slot, fr, arena)); }
    { HSS_PROF("set_slots", s); HSS_CUDA(launch_pdl(k_set_slots, dim3(cdiv(nse, 256)), dim3(256), 0, s, se, nse, elem_slot, 0)); }
    HSS_CHECK_LAUNCH("k_scatter_A");
    return HSS_OK;
}

template <class T>
int launch_gj_block_post(const BlockTile *tiles, int ntiles, const BlockJob *bjobs, const PanelJob *jobs,
                         const FrontDev *fr, T *arena, T *aold, const int *mws, cudaStream_t s) {
    if (ntiles == 0) return HSS_OK;
    HSS_PROF(sizeof(T) == 8 ? "gj_post_f64" : "gj_post_f32", s);
    HSS_CUDA(launch_pdl(k_gj_block_post<T>, dim3(ntiles), dim3(256), 0, s, tiles, bjobs, jobs, fr, arena, aold, mws));
    HSS_CHECK_LAUNCH("k_gj_block_post");
    return HSS_OK;
}

template <class T>
int launch_gj_post(const PanelTile *tiles, int ntiles, const PanelJob *jobs, const FrontDev *fr, T *arena, T *aold,
                   const T *xws, const int *mws, cudaStream_t s) {
    if (ntiles == 0) return HSS_OK;
    HSS_PROF(sizeof(T) == 8 ? "gj_post_f64" : "gj_post_f32", s);
    HSS_CUDA(launch_pdl(k_gj_post<T>, dim3(ntiles), dim3(256), 0, s, tiles, jobs, fr, arena, aold, xws, mws));
    HSS_CHECK_LAUNCH("k_gj_post");
    return HSS_OK;
}

template <class T, int KB, int R, int NT>
static cudaError_t launch_reg(const PanelJob *jobs, int njobs, size_t smem, const FrontDev *fr, T *arena, T *xws,
                              int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status,
                              cudaStream_t s) {
    return launch_pdl(k_gj_panel_reg<T, KB, R, NT>, dim3(njobs), dim3(NT), 0, s, jobs, fr, arena, xws, mws, piv, rperm, ilist,
                      iperm, status);
}

// Register panel for kb <= KB and rows <= R * NT: panels of at most 128 or 256
// rows run on that many threads (one row each: fewer warps at the per-pivot
// barriers), larger panels on PANEL_NT threads.
template <class T>
int launch_gj_panel_reg(const PanelJob *jobs, int njobs, int kb, int rows, const FrontDev *fr, T *arena, T *xws,
                        int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s,
                        double flops) {
    if (njobs == 0) return HSS_OK;
    HSS_PROF(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s, flops);
    const size_t smem = 0;   // the bookkeeping lives in registers
    cudaError_t e = cudaErrorInvalidValue;
    if (rows <= 2 * PANEL_SMALL_NT) {   // one row per thread on 128 or 256 threads
#define ONE(NT_)                                                                                                   \
    {                                                                                                              \
        if (kb <= 8)                                                                                               \
            e = launch_reg<T, 8, 1, NT_>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, \
                                         s);                                                                       \
        else if (kb <= 16)                                                                                         \
            e = launch_reg<T, 16, 1, NT_>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm,       \
                                          status, s);                                                              \
        else                                                                                                       \
            e = launch_reg<T, 32, 1, NT_>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm,       \
                                          status, s);                                                              \
    }
        if (rows <= PANEL_SMALL_NT)
            ONE(PANEL_SMALL_NT)
        else
            ONE(2 * PANEL_SMALL_NT)
#undef ONE
        if (e != cudaSuccess) return cuda_fail(e, "k_gj_panel_reg");
        return HSS_OK;
    }
    const int R = cdiv(rows, PANEL_NT);
#define REG(KB_, R_)                                                                                              \
    else if (kb <= KB_ && R <= R_) e = launch_reg<T, KB_, R_, PANEL_NT>(jobs, njobs, smem, fr, arena, xws, mws, piv, \
                                                                        rperm, ilist, iperm, status, s);
    if (false) {
    }
    REG(8, 1) REG(16, 1) REG(32, 1) REG(8, 2) REG(16, 2) REG(32, 2) REG(8, 3) REG(16, 3)
    REG(32, 3) REG(8, 4) REG(16, 4) REG(8, 6) REG(16, 6) REG(8, 8) REG(8, 12)
#undef REG
    if (e != cudaSuccess) return cuda_fail(e, "k_gj_panel_reg");
    return HSS_OK;
}

// Cluster panel for kb <= KB, rows <= R * NT * CL (NT = PANEL_NT): one
// cluster of CL CTAs per job.  Clusters of 16 are beyond the portable size and
// need the non-portable attribute; a configuration the GPU cannot place
// (cudaOccupancyMaxActiveClusters = 0) is reported as unusable.
template <class T, int KB, int R, int CL>
static cudaError_t launch_cl(const PanelJob *jobs, int njobs, size_t smem, const FrontDev *fr, T *arena, T *xws,
                             int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status,
                             cudaStream_t s) {
    auto kern = k_gj_panel_cl<T, KB, R, PANEL_NT, CL>;
    cudaError_t e = func_smem_once((const void *)kern, PANEL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    if (CL > 8 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(njobs * CL));
    cfg.blockDim = dim3(PANEL_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (njobs == 0) {   // placement query only
        int nc = 0;
        cfg.gridDim = dim3(CL);
        e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
        if (e != cudaSuccess) return e;
        return nc > 0 ? cudaSuccess : cudaErrorInvalidClusterSize;
    }
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see launch_pdl
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, jobs, fr, arena, xws, mws, piv, rperm, ilist, iperm, status);
}

// rows of a cluster panel step -> (R, CL): CL the smallest of 2, 4, 8, 16 with
// rows <= R PANEL_NT CL for R = 2 (FP32: 64 registers of panel values per
// thread; FP64: R = 1)
static void cl_shape(int rows, int tsize, int &R, int &CL) {
    R = tsize == 8 ? 1 : 2;
    for (CL = 2; CL < 16 && rows > R * PANEL_NT * CL; CL *= 2) {
    }
}

bool panel_cl_fits(int kb, int rows, int tsize) {
    if (kb != PANEL_KB_MAX) return false;
    int R, CL;
    cl_shape(rows, tsize, R, CL);
    if (rows > R * PANEL_NT * CL || 3L * rows * 4 > PANEL_SMEM_MAX) return false;
    // can the GPU place one cluster of this shape? (checked once per shape and device)
    static std::mutex mu;
    static int ok[2][5][64] = {};   // [tsize 4/8][log2 CL][device]: 0 unknown, 1 yes, -1 no
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return false;
    int lc = 0;
    while ((1 << lc) < CL) ++lc;
    std::lock_guard<std::mutex> lk(mu);
    int &st = ok[tsize == 8][lc][dev];
    if (st == 0) {
        cudaError_t e = cudaErrorInvalidValue;
        const size_t smem = 3 * (size_t)rows * 4;
        if (tsize == 8) {
            if (CL == 2) e = launch_cl<double, 32, 1, 2>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, nullptr, nullptr, nullptr);
            else if (CL == 4) e = launch_cl<double, 32, 1, 4>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr,
                                                              nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
            else if (CL == 8) e = launch_cl<double, 32, 1, 8>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr,
                                                              nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
            else e = launch_cl<double, 32, 1, 16>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr);
        } else {
            if (CL == 2) e = launch_cl<float, 32, 2, 2>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                         nullptr, nullptr, nullptr, nullptr, nullptr);
            else if (CL == 4) e = launch_cl<float, 32, 2, 4>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr,
                                                             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
            else if (CL == 8) e = launch_cl<float, 32, 2, 8>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr,
                                                             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
            else e = launch_cl<float, 32, 2, 16>(nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr, nullptr, nullptr, nullptr, nullptr);
        }
        if (e != cudaSuccess) cudaGetLastError();
        st = e == cudaSuccess ? 1 : -1;
    }
    return st > 0;
}

int panel_cl_capacity(int rows, int tsize) {
    int R, CL;
    cl_shape(rows, tsize, R, CL);
    return R * PANEL_NT * CL;
}

template <class T>
int launch_gj_panel_cl(const PanelJob *jobs, int njobs, int cap, size_t smem, const FrontDev *fr, T *arena, T *xws,
                       int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s,
                       double flops) {
    if (njobs == 0) return HSS_OK;
    int R, CL;
    cl_shape(cap, (int)sizeof(T), R, CL);
    HSS_PROF(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s, flops);
    cudaError_t e;
    if constexpr (sizeof(T) == 8) {
        if (CL == 2) e = launch_cl<T, 32, 1, 2>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else if (CL == 4) e = launch_cl<T, 32, 1, 4>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else if (CL == 8) e = launch_cl<T, 32, 1, 8>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else e = launch_cl<T, 32, 1, 16>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
    } else {
        if (CL == 2) e = launch_cl<T, 32, 2, 2>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else if (CL == 4) e = launch_cl<T, 32, 2, 4>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else if (CL == 8) e = launch_cl<T, 32, 2, 8>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
        else e = launch_cl<T, 32, 2, 16>(jobs, njobs, smem, fr, arena, xws, mws, piv, rperm, ilist, iperm, status, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "k_gj_panel_cl");
    return HSS_OK;
}

bool panel_reg_fits(int kb, int rows, int tsize) {
    const int R = cdiv(rows, PANEL_NT);
    // register budget of the panel rows: R * kb values of tsize bytes <= 96 32-bit registers
    if (R * kb * (tsize / 4) > 96) return false;
    if (3L * rows * 4 > PANEL_SMEM_MAX) return false;
    return (kb <= 32 && R <= 3) || (kb <= 16 && R <= 6) || (kb <= 8 && R <= 12);
}

template <class T>
int launch_gj_panel(const PanelJob *jobs, int njobs, size_t smem, const FrontDev *fr, T *arena, T *xws, int *mws,
                    int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s, double flops) {
    if (njobs == 0) return HSS_OK;
    HSS_SMEM(k_gj_panel<T>, PANEL_SMEM_MAX);
    HSS_PROF(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s, flops);
    HSS_CUDA(launch_pdl(k_gj_panel<T>, dim3(njobs), dim3(PANEL_NT), smem, s, jobs, fr, arena, xws, mws, piv, rperm, ilist,
                        iperm, status));
    HSS_CHECK_LAUNCH("k_gj_panel");
    return HSS_OK;
}

template int launch_scatter_A<double>(const hss_bsr *, const StageElem *, int, int *, const FrontDev *, double *,
                                      cudaStream_t);
template int launch_scatter_A<float>(const hss_bsr *, const StageElem *, int, int *, const FrontDev *, float *,
                                     cudaStream_t);
template int launch_gj_panel<double>(const PanelJob *, int, size_t, const FrontDev *, double *, double *, int *,
                                     int *, int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_panel<float>(const PanelJob *, int, size_t, const FrontDev *, float *, float *, int *, int *,
                                    int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_panel_cl<double>(const PanelJob *, int, int, size_t, const FrontDev *, double *, double *,
                                        int *, int *, int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_panel_cl<float>(const PanelJob *, int, int, size_t, const FrontDev *, float *, float *, int *,
                                       int *, int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_panel_reg<double>(const PanelJob *, int, int, int, const FrontDev *, double *, double *,
                                         int *, int *, int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_panel_reg<float>(const PanelJob *, int, int, int, const FrontDev *, float *, float *, int *,
                                        int *, int *, const int *, int *, int *, cudaStream_t, double);
template int launch_gj_block_post<double>(const BlockTile *, int, const BlockJob *, const PanelJob *,
                                          const FrontDev *, double *, double *, const int *, cudaStream_t);
template int launch_gj_block_post<float>(const BlockTile *, int, const BlockJob *, const PanelJob *,
                                         const FrontDev *, float *, float *, const int *, cudaStream_t);
template int launch_gj_post<double>(const PanelTile *, int, const PanelJob *, const FrontDev *, double *, double *,
                                    const double *, const int *, cudaStream_t);
template int launch_gj_post<float>(const PanelTile *, int, const PanelJob *, const FrontDev *, float *, float *,
                                   const float *, const int *, cudaStream_t);

}  // namespace hssnd
