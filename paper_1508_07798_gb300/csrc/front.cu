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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nse) elem_slot[se[i].elem] = value_is_index ? i : -1;
}

// ---------------------------------------------------------------- GJ panel
template <class T> struct ArgMax {
    T v;
    int i;
};

template <class T> __device__ ArgMax<T> block_argmax(ArgMax<T> x, ArgMax<T> *sh) {
    // largest |v|, ties to the lowest index
    for (int o = 16; o > 0; o >>= 1) {
        T v2 = __shfl_down_sync(0xffffffffu, x.v, o);
        int i2 = __shfl_down_sync(0xffffffffu, x.i, o);
        if (v2 > x.v || (v2 == x.v && i2 < x.i)) {
            x.v = v2;
            x.i = i2;
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        ArgMax<T> b = sh[0];
        for (int k = 1; k < nw; ++k)
            if (sh[k].v > b.v || (sh[k].v == b.v && sh[k].i < b.i)) b = sh[k];
        sh[0] = b;
    }
    __syncthreads();
    ArgMax<T> r = sh[0];
    __syncthreads();
    return r;
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
                                                    T *__restrict__ arena, T *__restrict__ aold_ws,
                                                    int *__restrict__ piv, int *__restrict__ rperm,
                                                    const int *__restrict__ ilist, int *__restrict__ iperm,
                                                    int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ ArgMax<T> red[PANEL_NT / 32];
    __shared__ T Xs[PANEL_KB_MAX * PANEL_KB_MAX];
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
        for (int c = 0; c < kb; ++c)
            for (int i = threadIdx.x; i < hT; i += PANEL_NT) P[i + ldp * c] = M[(k0 + i) + ld * (k0 + c)];
    } else {
        P = M + k0 + ld * k0;
        ldp = ld;
        rp = reinterpret_cast<int *>(smraw);
    }
    int *rglob = rperm + F.ioff;
    for (int i = threadIdx.x; i < hT; i += PANEL_NT) rp[i] = k0 == 0 ? i : rglob[k0 + i];
    __syncthreads();
    int *pv = piv + F.ioff;
    for (int j = 0; j < kb; ++j) {
        ArgMax<T> loc{T(-1), 0x7fffffff};
        for (int i = j + threadIdx.x; i < hT; i += PANEL_NT) {
            T a = fabs(P[i + ldp * j]);
            if (a > loc.v || (a == loc.v && i < loc.i)) {
                loc.v = a;
                loc.i = i;
            }
        }
        ArgMax<T> best = block_argmax(loc, red);
        int p = best.i;
        if (best.v == T(0)) {
            if (threadIdx.x == 0) atomicExch(&status[J.front], 1);
            p = j;
        }
        if (p != j)
            for (int c = threadIdx.x; c < kb; c += PANEL_NT) {
                T tmp = P[j + ldp * c];
                P[j + ldp * c] = P[p + ldp * c];
                P[p + ldp * c] = tmp;
            }
        if (threadIdx.x == 0) {
            pv[k0 + j] = k0 + p;
            swp[j] = p;
            int t = rp[j];
            rp[j] = rp[p];
            rp[p] = t;
        }
        __syncthreads();
        const T dinv = P[j + ldp * j] != T(0) ? T(1) / P[j + ldp * j] : T(0);
        for (int c = threadIdx.x; c < kb; c += PANEL_NT) rowj[c] = (c == j) ? T(0) : P[j + ldp * c] * dinv;
        __syncthreads();
        // eliminate column j from every other panel row (one thread per row)
        for (int i = threadIdx.x; i < hT; i += PANEL_NT) {
            if (i == j) continue;
            const T a = P[i + ldp * j];
            if (a != T(0)) {
#pragma unroll 8
                for (int c = 0; c < kb; ++c) P[i + ldp * c] -= a * rowj[c];
            }
            P[i + ldp * j] = -a * dinv;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kb; c += PANEL_NT) P[j + ldp * c] = (c == j) ? dinv : rowj[c];
        __syncthreads();
    }
    // X = inverse of the pivot block, kept for the rows outside the panel
    for (int q = threadIdx.x; q < kb * kb; q += PANEL_NT) {
        int i = q % kb, c = q / kb;
        Xs[i + kb * c] = P[i + ldp * c];
    }
    if (J.smem)
        for (int c = 0; c < kb; ++c)
            for (int i = threadIdx.x; i < hT; i += PANEL_NT) M[(k0 + i) + ld * (k0 + c)] = P[i + ldp * c];
    for (int i = threadIdx.x; i < hT; i += PANEL_NT) rglob[k0 + i] = rp[i];
    __syncthreads();
    // row swaps on the columns outside the panel, in pivot order (one thread per column)
    for (int c = threadIdx.x; c < n; c += PANEL_NT) {
        if (c >= k0 && c < k0 + kb) continue;
        T *col = M + ld * c + k0;
        for (int j = 0; j < kb; ++j) {
            int p = swp[j];
            if (p != j) {
                T tmp = col[j];
                col[j] = col[p];
                col[p] = tmp;
            }
        }
    }
    __syncthreads();
    // Aold: the (swapped) pivot rows over all columns
    T *Ao = aold_ws + J.aoff;
    for (int q = threadIdx.x; q < kb * n; q += PANEL_NT) {
        int i = q % kb, c = q / kb;
        Ao[i + (long)kb * c] = M[(k0 + i) + ld * c];
    }
    // rows outside [k0, ni): F(i, P) <- -F(i, P) X
    int nout = n - hT;
    for (int r = threadIdx.x; r < nout; r += PANEL_NT) {
        int i = r < k0 ? r : r + hT;
        T old[PANEL_KB_MAX];
#pragma unroll
        for (int s = 0; s < PANEL_KB_MAX; ++s)
            if (s < kb) old[s] = M[i + ld * (k0 + s)];
        for (int c = 0; c < kb; ++c) {
            T acc = T(0);
#pragma unroll
            for (int s = 0; s < PANEL_KB_MAX; ++s)
                if (s < kb) acc = fma(old[s], Xs[s + kb * c], acc);
            M[i + ld * (k0 + c)] = -acc;
        }
    }
    // last panel: gather list of the apply
    if (k0 + kb == ni) {
        __syncthreads();
        for (int j = threadIdx.x; j < ni; j += PANEL_NT) {
            int r = j < k0 ? rglob[j] : rp[j - k0];
            iperm[F.iperm_off + j] = ilist[F.iset_off + r];
        }
    }
}

// ---------------------------------------------------------------- launchers
template <class T>
int launch_scatter_A(const hss_bsr *A, const StageElem *se, int nse, int *elem_slot, const FrontDev *fr, T *arena,
                     cudaStream_t s) {
    if (nse == 0) return HSS_OK;
    { HSS_PROF("set_slots", s); k_set_slots<<<cdiv(nse, 256), 256, 0, s>>>(se, nse, elem_slot, 1); }
    { HSS_PROF("scatter_A", s);
    k_scatter_A<T><<<cdiv((long)nse * 32, 256), 256, 0, s>>>(A->row_ptr, A->col_idx, A->val, A->bs, se, nse,
                                                             elem_slot, fr, arena); }
    { HSS_PROF("set_slots", s); k_set_slots<<<cdiv(nse, 256), 256, 0, s>>>(se, nse, elem_slot, 0); }
    HSS_CHECK_LAUNCH("k_scatter_A");
    return HSS_OK;
}

template <class T>
int launch_gj_panel(const PanelJob *jobs, int njobs, size_t smem, const FrontDev *fr, T *arena, T *aold, int *piv,
                    int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s) {
    if (njobs == 0) return HSS_OK;
    static bool configured[2] = {false, false};
    int ti = sizeof(T) == 8 ? 0 : 1;
    if (!configured[ti]) {
        cudaFuncSetAttribute(k_gj_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_MAX);
        configured[ti] = true;
    }
    HSS_PROF(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s);
    k_gj_panel<T><<<njobs, PANEL_NT, smem, s>>>(jobs, fr, arena, aold, piv, rperm, ilist, iperm, status);
    HSS_CHECK_LAUNCH("k_gj_panel");
    return HSS_OK;
}

template int launch_scatter_A<double>(const hss_bsr *, const StageElem *, int, int *, const FrontDev *, double *,
                                      cudaStream_t);
template int launch_scatter_A<float>(const hss_bsr *, const StageElem *, int, int *, const FrontDev *, float *,
                                     cudaStream_t);
template int launch_gj_panel<double>(const PanelJob *, int, size_t, const FrontDev *, double *, double *, int *,
                                     int *, const int *, int *, int *, cudaStream_t);
template int launch_gj_panel<float>(const PanelJob *, int, size_t, const FrontDev *, float *, float *, int *, int *,
                                    const int *, int *, int *, cudaStream_t);

}  // namespace hssnd
