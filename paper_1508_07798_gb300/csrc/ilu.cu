// Block ILU(0) on the BSR pattern of A: the comparison preconditioner of
// Sec. 5 ("a standard ILU preconditioner"; zero fill, natural element order).
//
//   factor, row form of Gaussian elimination, for every block row i:
//       for each stored k < i, ascending:   L_ik = A_ik U_kk^-1
//           for each stored (k, j), j > k, that row i also stores:   A_ij -= L_ik U_kj
//       U_ii^-1 by Gauss-Jordan with partial pivoting (kept for the sweeps)
//   apply, y = U^-1 L^-1 x:
//       forward:   y_i = x_i - sum_{k<i} L_ik y_k
//       backward:  y_i = U_ii^-1 (y_i - sum_{j>i} U_ij y_j)
//
// Row i depends on the rows of its stored lower (forward) / upper (backward)
// blocks only, so rows are grouped into levels (a row's level is one more than
// the highest level it depends on) and each level is one launch: one CTA per
// row in the factorization, one warp per row in the sweeps.  The sweeps are
// captured once per handle into a CUDA graph.
#include "internal.h"
#include "factor.h"
#include "prof.h"

#include <algorithm>

namespace hssnd {

constexpr int ILU_NT = 128;          // factorization: threads per CTA (one block row)
constexpr int ILU_MAX_BS = 64;
constexpr int ILU_AP_NT = 128;       // sweeps: one warp per block row
constexpr int ILU_AP_WPB = ILU_AP_NT / 32;
constexpr int ILU_RB = 8;            // right-hand sides per sweep of the multi-RHS graph

struct IluParams {
    const double *x;
    long ldx;
    double *y;
    long ldy;
    int nrhs;
};

// One CTA per block row of the level.  Shared memory: L_ik (bs x bs), the
// augmented [U_ii | I] (bs x 2bs) and one column of factors (bs).
__global__ void __launch_bounds__(ILU_NT) k_ilu_row(const int *__restrict__ rows, int bs,
                                                    const int *__restrict__ rowptr, const int *__restrict__ colidx,
                                                    const int *__restrict__ diag, const int *__restrict__ upd_off,
                                                    const int2 *__restrict__ upd, double *__restrict__ lu,
                                                    double *__restrict__ dinv, int *__restrict__ status) {
    extern __shared__ double sm[];
    const int i = rows[blockIdx.x];
    const int bb = bs * bs, w2 = 2 * bs;
    double *L = sm;
    double *G = sm + bb;
    double *fcol = G + bs * w2;
    __shared__ int piv;
    __shared__ double pval;
    for (int q = rowptr[i]; q < diag[i]; ++q) {
        const int k = colidx[q];
        double *Aik = lu + (long)q * bb;
        const double *Dk = dinv + (long)k * bb;
        for (int e = threadIdx.x; e < bb; e += blockDim.x) {
            const int r = e / bs, c = e - r * bs;
            double acc = 0.0;
            for (int t = 0; t < bs; ++t) acc = fma(Aik[r * bs + t], Dk[t * bs + c], acc);
            L[e] = acc;
        }
        __syncthreads();   // every product read A_ik before it is overwritten
        for (int e = threadIdx.x; e < bb; e += blockDim.x) Aik[e] = L[e];
        const int u0 = upd_off[q], tot = (upd_off[q + 1] - u0) * bb;
        for (int g = threadIdx.x; g < tot; g += blockDim.x) {
            const int u = u0 + g / bb, e = g % bb;
            const int r = e / bs, c = e - r * bs;
            const int2 qq = upd[u];   // x: stored block (k, j); y: stored block (i, j)
            const double *Ukj = lu + (long)qq.x * bb;
            double acc = 0.0;
            for (int t = 0; t < bs; ++t) acc = fma(L[r * bs + t], Ukj[t * bs + c], acc);
            lu[(long)qq.y * bb + e] -= acc;
        }
        __syncthreads();   // the updated blocks of row i are read by the next k
    }
    // U_ii^-1: Gauss-Jordan on [U_ii | I], pivot = largest |entry| of the column (lowest row on ties)
    const double *Aii = lu + (long)diag[i] * bb;
    for (int e = threadIdx.x; e < bs * w2; e += blockDim.x) {
        const int r = e / w2, c = e - r * w2;
        G[e] = c < bs ? Aii[r * bs + c] : (c - bs == r ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < bs; ++j) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = j;
            for (int r = j + (int)threadIdx.x; r < bs; r += 32) {
                const double v = fabs(G[r * w2 + j]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_down_sync(0xffffffffu, best, o);
                const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) {
                    best = v2;
                    bi = i2;
                }
            }
            if (threadIdx.x == 0) {
                piv = bi;
                pval = G[bi * w2 + j];
            }
        }
        __syncthreads();
        const int pr = piv;
        const double p = pval;
        if (p == 0.0) {   // uniform: every thread read the same shared value
            if (threadIdx.x == 0) atomicCAS(status, 0, i + 1);
            return;
        }
        if (pr != j)
            for (int c = threadIdx.x; c < w2; c += blockDim.x) {
                const double t = G[j * w2 + c];
                G[j * w2 + c] = G[pr * w2 + c];
                G[pr * w2 + c] = t;
            }
        __syncthreads();
        for (int c = threadIdx.x; c < w2; c += blockDim.x) G[j * w2 + c] /= p;
        for (int r = threadIdx.x; r < bs; r += blockDim.x) fcol[r] = G[r * w2 + j];
        __syncthreads();
        for (int e = threadIdx.x; e < bs * w2; e += blockDim.x) {
            const int r = e / w2, c = e - r * w2;
            if (r != j) G[e] = fma(-fcol[r], G[j * w2 + c], G[e]);
        }
        __syncthreads();
    }
    double *Di = dinv + (long)i * bb;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const int r = e / bs, c = e - r * bs;
        Di[e] = G[r * w2 + bs + c];
    }
}

// Forward sweep over one level: y_i = x_i - sum_{k<i} L_ik y_k.  One warp per
// block row, lane = component (two passes when bs > 32).
template <int RB>
__global__ void __launch_bounds__(ILU_AP_NT) k_ilu_fwd(const int *__restrict__ rows, int nrows, int bs,
                                                       const int *__restrict__ rowptr, const int *__restrict__ colidx,
                                                       const int *__restrict__ diag, const double *__restrict__ lu,
                                                       const IluParams *__restrict__ prm) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * ILU_AP_WPB + (threadIdx.x >> 5);
    if (w >= nrows) return;
    const int i = rows[w];
    const double *x = prm->x;
    double *y = prm->y;
    const long ldx = prm->ldx, ldy = prm->ldy;
    const int nrhs = prm->nrhs, bb = bs * bs;
    for (int c0 = 0; c0 < bs; c0 += 32) {
        const int comp = c0 + lane;
        if (comp >= bs) break;
        double acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = r < nrhs ? x[(long)i * bs + comp + ldx * r] : 0.0;
        for (int q = rowptr[i]; q < diag[i]; ++q) {
            const long kb = (long)colidx[q] * bs;
            const double *Lr = lu + (long)q * bb + (long)comp * bs;
            for (int t = 0; t < bs; ++t) {
                const double m = Lr[t];
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (r < nrhs) acc[r] = fma(-m, y[kb + t + ldy * r], acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r < nrhs) y[(long)i * bs + comp + ldy * r] = acc[r];
    }
}

// Backward sweep over one level: t = y_i - sum_{j>i} U_ij y_j, y_i = U_ii^-1 t.
template <int RB>
__global__ void __launch_bounds__(ILU_AP_NT) k_ilu_bwd(const int *__restrict__ rows, int nrows, int bs,
                                                       const int *__restrict__ rowptr, const int *__restrict__ colidx,
                                                       const int *__restrict__ diag, const double *__restrict__ lu,
                                                       const double *__restrict__ dinv,
                                                       const IluParams *__restrict__ prm) {
    __shared__ double tsh[ILU_AP_WPB][ILU_MAX_BS * RB];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int w = blockIdx.x * ILU_AP_WPB + wl;
    if (w >= nrows) return;   // whole warps leave together; no block-wide barrier below
    const int i = rows[w];
    double *y = prm->y;
    const long ldy = prm->ldy;
    const int nrhs = prm->nrhs, bb = bs * bs;
    double *t = tsh[wl];
    for (int comp = lane; comp < bs; comp += 32) {
        double acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = r < nrhs ? y[(long)i * bs + comp + ldy * r] : 0.0;
        for (int q = diag[i] + 1; q < rowptr[i + 1]; ++q) {
            const long jb = (long)colidx[q] * bs;
            const double *Ur = lu + (long)q * bb + (long)comp * bs;
            for (int c = 0; c < bs; ++c) {
                const double m = Ur[c];
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (r < nrhs) acc[r] = fma(-m, y[jb + c + ldy * r], acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) t[r * bs + comp] = acc[r];
    }
    __syncwarp();
    const double *Di = dinv + (long)i * bb;
    for (int comp = lane; comp < bs; comp += 32) {
        double acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = 0.0;
        for (int c = 0; c < bs; ++c) {
            const double m = Di[comp * bs + c];
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[r] = fma(m, t[r * bs + c], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r < nrhs) y[(long)i * bs + comp + ldy * r] = acc[r];
    }
}

__global__ void k_ilu_set(IluParams *d, IluParams v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d = v;
}

}  // namespace hssnd

struct hss_ilu_t {
    int nb = 0, bs = 0;
    long ndof = 0, nnzb = 0;
    hssnd::DevBuf d_lu, d_dinv, d_rowptr, d_colidx, d_diag, d_frows, d_brows, d_params;
    std::vector<int> foff, boff;   // level offsets into the forward / backward row lists
    double bytes_per_sweep = 0;    // factor bytes read by one apply (L, U and the U_ii^-1)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_kernels[2] = {0, 0};
    ~hss_ilu_t() {
        for (auto &g : gexec)
            if (g) cudaGraphExecDestroy(g);
    }
};

namespace hssnd {

long ilu_ndof(const hss_ilu_t *M) { return M ? M->ndof : -1; }

template <int RB> static int record_ilu(const hss_ilu_t *M, cudaStream_t s, int &nk) {
    const IluParams *prm = M->d_params.as<IluParams>();
    const int *rp = M->d_rowptr.as<int>(), *ci = M->d_colidx.as<int>(), *dg = M->d_diag.as<int>();
    const double *lu = M->d_lu.as<double>(), *di = M->d_dinv.as<double>();
    nk = 0;
    for (size_t l = 0; l + 1 < M->foff.size(); ++l) {
        const int n = M->foff[l + 1] - M->foff[l];
        k_ilu_fwd<RB><<<cdiv(n, ILU_AP_WPB), ILU_AP_NT, 0, s>>>(M->d_frows.as<int>() + M->foff[l], n, M->bs, rp, ci,
                                                                dg, lu, prm);
        ++nk;
    }
    for (size_t l = 0; l + 1 < M->boff.size(); ++l) {
        const int n = M->boff[l + 1] - M->boff[l];
        k_ilu_bwd<RB><<<cdiv(n, ILU_AP_WPB), ILU_AP_NT, 0, s>>>(M->d_brows.as<int>() + M->boff[l], n, M->bs, rp, ci,
                                                                dg, lu, di, prm);
        ++nk;
    }
    HSS_CHECK_LAUNCH("ilu sweeps");
    return HSS_OK;
}

static int build_ilu_graph(hss_ilu_t *M, int slot) {
    cudaStream_t cs;
    HSS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    int rc = HSS_OK;
    prof_set_capture(true);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int nk = 0;
        rc = slot == 0 ? record_ilu<1>(M, cs, nk) : record_ilu<ILU_RB>(M, cs, nk);
        e = cudaStreamEndCapture(cs, &g);
        M->graph_kernels[slot] = nk;
    }
    prof_set_capture(false);
    if (e == cudaSuccess && rc == HSS_OK) e = cudaGraphInstantiate(&M->gexec[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "ilu0 graph");
    return HSS_OK;
}

int ilu_apply(const hss_ilu_t *M, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s) {
    hss_ilu_t *mm = const_cast<hss_ilu_t *>(M);
    const int slot = nrhs == 1 ? 0 : 1;
    int rc;
    if (!M->gexec[slot] && (rc = build_ilu_graph(mm, slot))) return rc;
    HSS_PROF("ilu0_apply", s, M->bytes_per_sweep + 4.0 * 8.0 * M->ndof * nrhs);
    for (int k = 0; k < nrhs; k += ILU_RB) {   // one sweep pair per block of up to ILU_RB right-hand sides
        IluParams pv{x + ldx * k, ldx, y + ldy * k, ldy, std::min(ILU_RB, nrhs - k)};
        prof_add_launches(M->graph_kernels[slot]);
        k_ilu_set<<<1, 32, 0, s>>>(mm->d_params.as<IluParams>(), pv);
        HSS_CHECK_LAUNCH("k_ilu_set");
        HSS_CUDA(cudaGraphLaunch(M->gexec[slot], s));
    }
    return HSS_OK;
}

// Rows grouped by level: lev[i] from the rows i depends on; returns the rows
// sorted by level (ascending row id inside a level) and the level offsets.
static void levels(int nb, const std::vector<int> &lev, std::vector<int> &rows, std::vector<int> &off) {
    int nl = 0;
    for (int v : lev) nl = std::max(nl, v + 1);
    off.assign(nl + 1, 0);
    for (int v : lev) off[v + 1]++;
    for (int l = 0; l < nl; ++l) off[l + 1] += off[l];
    std::vector<int> fill(off.begin(), off.end() - 1);
    rows.assign(nb, 0);
    for (int i = 0; i < nb; ++i) rows[fill[lev[i]]++] = i;
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int ilu0_factor(const hss_bsr *A, void *stream, hss_ilu_t **out) {
    if (!out) {
        set_error("ilu0_factor: null output handle");
        return HSS_EINVAL;
    }
    *out = nullptr;
    if (!A || A->nb < 1 || A->bs < 1 || A->bs > ILU_MAX_BS || !A->row_ptr || !A->col_idx || !A->val) {
        set_error("ilu0_factor: invalid matrix (null pointers, or block size outside [1, 64])");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = A->nb, bs = A->bs;
    std::vector<int> rp(nb + 1);
    HSS_CUDA(cudaMemcpyAsync(rp.data(), A->row_ptr, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    const long nnzb = rp[nb];
    if (rp[0] != 0 || nnzb < nb) {
        set_error("ilu0_factor: invalid row pointers");
        return HSS_EINVAL;
    }
    std::vector<int> ci(nnzb);
    HSS_CUDA(cudaMemcpyAsync(ci.data(), A->col_idx, sizeof(int) * nnzb, cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    // structure checks, diagonal positions, levels
    std::vector<int> dg(nb, -1), flev(nb, 0), blev(nb, 0);
    for (int i = 0; i < nb; ++i) {
        if (rp[i + 1] < rp[i]) {
            set_error("ilu0_factor: invalid row pointers");
            return HSS_EINVAL;
        }
        for (int q = rp[i]; q < rp[i + 1]; ++q) {
            if (ci[q] < 0 || ci[q] >= nb || (q > rp[i] && ci[q] <= ci[q - 1])) {
                set_error("ilu0_factor: block columns must be in range and strictly ascending per row");
                return HSS_EINVAL;
            }
            if (ci[q] == i) dg[i] = q;
        }
        if (dg[i] < 0) {
            set_error("ilu0_factor: block row " + std::to_string(i) + " stores no diagonal block");
            return HSS_EINVAL;
        }
    }
    for (int i = 0; i < nb; ++i)
        for (int q = rp[i]; q < dg[i]; ++q) flev[i] = std::max(flev[i], flev[ci[q]] + 1);
    for (int i = nb - 1; i >= 0; --i)
        for (int q = dg[i] + 1; q < rp[i + 1]; ++q) blev[i] = std::max(blev[i], blev[ci[q]] + 1);
    // trailing updates of each stored lower block (i, k): pairs (block (k, j), block (i, j)), j > k
    std::vector<int> uoff(nnzb + 1, 0);
    std::vector<int2> upd;
    for (int i = 0; i < nb; ++i) {
        for (int q = rp[i]; q < rp[i + 1]; ++q) {
            uoff[q] = (int)upd.size();
            if (q >= dg[i]) continue;
            const int k = ci[q];
            int a = dg[k] + 1, b = q + 1;   // merge row k's upper part with row i's columns after k
            while (a < rp[k + 1] && b < rp[i + 1]) {
                if (ci[a] == ci[b]) upd.push_back(make_int2(a++, b++));
                else if (ci[a] < ci[b]) ++a;
                else ++b;
            }
        }
    }
    uoff[nnzb] = (int)upd.size();
    std::vector<int> frows, foff, brows, boff;
    levels(nb, flev, frows, foff);
    levels(nb, blev, brows, boff);

    hss_ilu_t *M = new hss_ilu_t();
    M->nb = nb;
    M->bs = bs;
    M->ndof = (long)nb * bs;
    M->nnzb = nnzb;
    M->foff = foff;
    M->boff = boff;
    M->bytes_per_sweep = 8.0 * ((double)nnzb + nb) * bs * bs;
    const size_t bb = (size_t)bs * bs;
    DevBuf d_uoff, d_upd, d_status;
    int rc;
    if ((rc = M->d_lu.alloc(sizeof(double) * bb * nnzb)) || (rc = M->d_dinv.alloc(sizeof(double) * bb * nb)) ||
        (rc = upload(M->d_rowptr, rp, s)) || (rc = upload(M->d_colidx, ci, s)) || (rc = upload(M->d_diag, dg, s)) ||
        (rc = upload(M->d_frows, frows, s)) || (rc = upload(M->d_brows, brows, s)) ||
        (rc = M->d_params.alloc(sizeof(IluParams))) || (rc = upload(d_uoff, uoff, s)) ||
        (rc = upload(d_upd, upd, s)) || (rc = d_status.alloc(sizeof(int)))) {
        delete M;
        return rc;
    }
    auto fail = [&](int code) {
        delete M;
        return code;
    };
    if (cudaMemcpyAsync(M->d_lu.p, A->val, sizeof(double) * bb * nnzb, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(d_status.p, 0, sizeof(int), s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "ilu0_factor copy"));
    const size_t smem = sizeof(double) * (bb + 2 * bb + bs);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ilu_row, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "ilu0_factor smem"));
    for (size_t l = 0; l + 1 < foff.size(); ++l) {
        const int n = foff[l + 1] - foff[l];
        HSS_PROF("ilu0_factor", s);
        k_ilu_row<<<n, ILU_NT, smem, s>>>(M->d_frows.as<int>() + foff[l], bs, M->d_rowptr.as<int>(),
                                         M->d_colidx.as<int>(), M->d_diag.as<int>(), d_uoff.as<int>(),
                                         d_upd.as<int2>(), M->d_lu.as<double>(), M->d_dinv.as<double>(),
                                         d_status.as<int>());
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(cuda_fail(e, "k_ilu_row"));
    }
    int st = 0;
    if (cudaMemcpyAsync(&st, d_status.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "ilu0_factor status"));
    if (st) {
        set_error("ilu0_factor: singular diagonal block of U in block row " + std::to_string(st - 1));
        return fail(HSS_ESINGULAR);
    }
    *out = M;
    return HSS_OK;
}

extern "C" int ilu0_apply(const hss_ilu_t *M, int nrhs, const double *x, int ldx, double *y, int ldy, void *stream) {
    if (!M || !x || !y || nrhs < 0 || ldx < M->ndof || ldy < M->ndof) {
        set_error("ilu0_apply: invalid argument");
        return HSS_EINVAL;
    }
    if (nrhs == 0) return HSS_OK;
    return ilu_apply(M, nrhs, x, ldx, y, ldy, (cudaStream_t)stream);
}

extern "C" void ilu0_destroy(hss_ilu_t *M) { delete M; }
