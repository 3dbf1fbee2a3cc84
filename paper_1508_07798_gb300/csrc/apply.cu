// hss_apply: y = M^-t D^-1 L^-1 x (end of Sec. 4.2), level by level.
//
// After the Gauss-Jordan sweep every front holds [F_ii^-1 P^t ; -F_bi F_ii^-1 P^t]
// in its I columns and W = F_ii^-1 F_ib in the top-right block, so
//   forward  (deepest level first, then the top block):
//       z = x(Iperm);  t = F_ii^-1 x_I = rows [0,ni) of [..] z;  x_B += rows [ni,n) of [..] z
//   backward (top block first, then down to the leaves):
//       x_I = t - W x_B
// t is parked in a second vector so that all row tiles of a front read the
// same x_I.  Fronts of one level touch disjoint dofs, so one launch per level
// covers all of them; each CTA handles APPLY_ROWS rows of one front.
#include "internal.h"
#include "front.h"
#include "factor.h"
#include "prof.h"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

namespace hssnd {

constexpr int AP_NT = 256;
constexpr int AP_RG = AP_NT / APPLY_ROWS;   // column groups per CTA
constexpr int AP_ZC = 1024;                  // z entries staged per chunk (per right-hand side block)

// One cluster of `cs` CTAs per row tile of one front; CTA rank r multiplies the
// tile's rows by its 1/cs share of the columns, the partial sums meet in the
// rank-0 CTA's registers through distributed shared memory (fixed order).
//   FWD: y = [F_ii^-1 P^t ; -F_bi F_ii^-1 P^t] x(Iperm)  ->  t = y[0,ni), x_B += y[ni,n)
//   BWD: x_I = t - W x_B
template <class T, int RB, bool FWD>
__global__ void __launch_bounds__(AP_NT) k_apply(const ApplyTile *__restrict__ tiles, const FrontDev *__restrict__ fr,
                                               const T *__restrict__ arena, const int *__restrict__ iperm,
                                               const int *__restrict__ ilist, const int *__restrict__ blist,
                                               const ApplyParams *__restrict__ prm) {
    double *__restrict__ w = prm->w;
    const long ldw = prm->ldw;
    double *__restrict__ tv = prm->tv;
    const long ldt = prm->ldt;
    const int nrhs = prm->nrhs;
    __shared__ double zs[AP_ZC * RB];
    __shared__ double red[AP_RG][APPLY_ROWS][RB];
    __shared__ double part[RB][APPLY_ROWS];
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
    const ApplyTile tl = tiles[blockIdx.x / cs];
    const FrontDev F = fr[tl.front];
    const T *M = arena + F.foff;
    const int ncols = FWD ? F.ni : F.nb, colbase = FWD ? 0 : F.ni, nrows = FWD ? F.n : F.ni;
    const int chunk = (ncols + cs - 1) / cs;
    const int c_lo = min(ncols, crank * chunk), c_hi = min(ncols, c_lo + chunk);
    const int tx = threadIdx.x % APPLY_ROWS, ty = threadIdx.x / APPLY_ROWS;
    const int i = tl.row0 + tx;
    for (int rb0 = 0; rb0 < nrhs; rb0 += RB) {
        double acc[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) acc[q] = 0.0;
        for (int c0 = c_lo; c0 < c_hi; c0 += AP_ZC) {
            const int cn = min(AP_ZC, c_hi - c0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < cn * RB; idx += AP_NT) {
                int c = idx % cn, q = idx / cn;
                int rr = rb0 + q;
                int dof = FWD ? iperm[F.iperm_off + c0 + c] : blist[F.bset_off + c0 + c];
                zs[c + AP_ZC * q] = rr < nrhs ? w[dof + ldw * rr] : 0.0;
            }
            __syncthreads();
            if (i < nrows) {
                const T *col = M + i + (long)F.n * (colbase + c0);
#pragma unroll 8
                for (int c = ty; c < cn; c += AP_RG) {
                    double m = (double)col[(long)F.n * c];
#pragma unroll
                    for (int q = 0; q < RB; ++q) acc[q] = fma(m, zs[c + AP_ZC * q], acc[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) red[ty][tx][q] = acc[q];
        __syncthreads();
        if (ty == 0) {
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                double y = 0.0;
                for (int g = 0; g < AP_RG; ++g) y += red[g][tx][q];
                part[q][tx] = y;
            }
        }
        cl.sync();
        if (crank == 0 && ty == 0 && i < nrows) {
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                int rr = rb0 + q;
                if (rr >= nrhs) break;
                double y = 0.0;
                for (int r = 0; r < cs; ++r) y += cl.map_shared_rank(&part[q][0], r)[tx];
                if (FWD) {
                    if (i < F.ni)
                        tv[ilist[F.iset_off + i] + ldt * rr] = y;
                    else
                        w[blist[F.bset_off + i - F.ni] + ldw * rr] += y;
                } else {
                    int dof = ilist[F.iset_off + i];
                    w[dof + ldw * rr] = tv[dof + ldt * rr] - y;
                }
            }
        }
        cl.sync();
    }
}

__global__ void k_apply_set(ApplyParams *d, ApplyParams v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d = v;
}

// w = x (every right-hand side), skipped when they alias
__global__ void k_apply_copyin(const ApplyParams *__restrict__ prm, long N) {
    const double *x = prm->x;
    double *w = prm->w;
    if (x == w) return;
    long tot = N * prm->nrhs;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < tot; g += (long)gridDim.x * blockDim.x) {
        long r = g / N, i = g % N;
        w[i + prm->ldw * r] = x[i + prm->ldx * r];
    }
}

template <class T, int RB, bool FWD>
static cudaError_t launch_apply(int ntiles, int cs, cudaStream_t s, const ApplyTile *tiles, const FrontDev *fr,
                                const T *arena, const int *iperm, const int *ilist, const int *blist,
                                const ApplyParams *prm) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntiles * cs);
    cfg.blockDim = dim3(AP_NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_apply<T, RB, FWD>, tiles, fr, arena, iperm, ilist, blist, prm);
}

// The whole sweep (copy-in, forward levels, top block, backward levels) as
// one kernel sequence on stream s; parameters come from f->d_aparams.
template <class T, int RB> static int record_sweep(const hss_factor_t *f, cudaStream_t s, int &nk) {
    const T *arena = f->arena_ptr<T>();
    const ApplyParams *prm = f->d_aparams.as<ApplyParams>();
    nk = 0;
    k_apply_copyin<<<2 * 152, 256, 0, s>>>(prm, f->ndof);
    ++nk;
    for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        for (size_t q = 0; q < f->apply.size(); ++q) {
            const ApplyStage &st = fwd ? f->apply[q] : f->apply[f->apply.size() - 1 - q];
            const int *ilist = st.top ? f->d_topset.as<int>() : f->tree->d_iset.as<int>();
            const int nt = fwd ? st.nfwd : st.nbwd;
            if (nt == 0) continue;
            cudaError_t e = fwd ? launch_apply<T, RB, true>(nt, st.cs_fwd, s, st.d_fwd, st.d_fronts, arena,
                                                              f->d_iperm.as<int>(), ilist, f->tree->d_bset.as<int>(), prm)
                                : launch_apply<T, RB, false>(nt, st.cs_bwd, s, st.d_bwd, st.d_fronts, arena,
                                                               f->d_iperm.as<int>(), ilist, f->tree->d_bset.as<int>(), prm);
            if (e != cudaSuccess) return cuda_fail(e, "k_apply launch");
            ++nk;
        }
    }
    HSS_CHECK_LAUNCH("apply sweep");
    return HSS_OK;
}

template <class T> static int build_graph(hss_factor_t *f, int slot) {
    cudaStream_t cs;
    HSS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    int rc = HSS_OK;
    prof_set_capture(true);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int nk = 0;
        rc = slot == 0 ? record_sweep<T, 1>(f, cs, nk) : record_sweep<T, 4>(f, cs, nk);
        e = cudaStreamEndCapture(cs, &g);
        f->graph_kernels[slot] = nk;
    }
    prof_set_capture(false);
    if (e == cudaSuccess && rc == HSS_OK) e = cudaGraphInstantiate(&f->gexec[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "apply graph");
    return HSS_OK;
}

int apply_factor(const hss_factor_t *f, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s) {
    hss_factor_t *mf = const_cast<hss_factor_t *>(f);
    int rc;
    if ((rc = mf->tvec.alloc(sizeof(double) * (size_t)f->ndof * nrhs))) return rc;
    if ((rc = mf->d_aparams.alloc(sizeof(ApplyParams)))) return rc;
    const int slot = nrhs == 1 ? 0 : 1;
    if (!f->gexec[slot]) {
        rc = f->precision == HSS_FP32 ? build_graph<float>(mf, slot) : build_graph<double>(mf, slot);
        if (rc) return rc;
    }
    ApplyParams pv{x, ldx, y, ldy, mf->tvec.as<double>(), (long)f->ndof, nrhs};
    HSS_PROF("apply", s, f->apply_bytes(nrhs));
    prof_add_launches(f->graph_kernels[slot]);
    k_apply_set<<<1, 32, 0, s>>>(mf->d_aparams.as<ApplyParams>(), pv);
    HSS_CHECK_LAUNCH("k_apply_set");
    HSS_CUDA(cudaGraphLaunch(f->gexec[slot], s));
    return HSS_OK;
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_apply(const hss_factor_t *f, int nrhs, const double *x, int ldx, double *y, int ldy,
                         void *stream) {
    if (!f || !x || !y || nrhs < 0 || ldx < f->ndof || ldy < f->ndof) {
        set_error("hss_apply: invalid argument");
        return HSS_EINVAL;
    }
    if (nrhs == 0) return HSS_OK;
    return apply_factor(f, nrhs, x, ldx, y, ldy, (cudaStream_t)stream);
}
