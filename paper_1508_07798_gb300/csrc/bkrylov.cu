// Batched right-preconditioned flexible GMRES over a forest factor
// (hss_factor_batched): one independent Krylov process per (instance,
// right-hand side), all advanced in lock step so that every Arnoldi step costs
// one preconditioner apply and one SpMV over the whole batch.
//
// A process owns rows [inst_dof[i], inst_dof[i + 1]) of one column of the
// N x nrhs block vectors.  Inner products and vector updates run over chunks
// of at most BK_CHUNK rows of one process; partial sums are reduced per
// process in a fixed order (deterministic).  Processes that have converged,
// or that stopped for this restart cycle, are masked by an activity flag and
// left untouched.  The algorithm per process is the one of fgmres_solve:
// classical Gram-Schmidt applied twice, Givens rotations on the device, a true
// FP64 residual at each restart.
#include <cmath>

#include "factor.h"
#include "prof.h"

namespace hssnd {
namespace {

constexpr int BK_NT = 256;
constexpr int BK_CHUNK = 4096;
constexpr int BK_MAXM = 32;   // largest restart length + 1

struct BChunk {
    int p;          // process
    int col;        // its column
    int row0, len;  // rows [row0, row0 + len) of the block vectors
};

struct BProc {
    int col, row0, len;
    int c0, c1;     // its chunks [c0, c1)
};

// partial[c * BK_MAXM + q] = sum over chunk c of V_q(rows, col) * w(rows, col), q < nq.
// V_q = V + q * vstride, element (row, col) at col * ldv + row; w likewise with ldw.
__global__ void k_bdots(const double *__restrict__ V, long ldv, long vstride, int nq, const double *__restrict__ w,
                        long ldw, const BChunk *__restrict__ ch, const int *__restrict__ act,
                        double *__restrict__ partial) {
    const BChunk C = ch[blockIdx.x];
    if (!act[C.p]) return;
    __shared__ double sh[BK_NT / 32][BK_MAXM + 1];
    double acc[BK_MAXM];
#pragma unroll
    for (int q = 0; q < BK_MAXM; ++q) acc[q] = 0.0;
    const double *wc = w + (long)C.col * ldw + C.row0;
    const double *vc = V + (long)C.col * ldv + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) {
        const double wi = wc[i];
#pragma unroll
        for (int q = 0; q < BK_MAXM; ++q)
            if (q < nq) acc[q] = fma(vc[i + vstride * q], wi, acc[q]);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < BK_MAXM; ++q) {
        if (q >= nq) break;
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += BK_NT) {
        double s = 0.0;
        for (int k = 0; k < BK_NT / 32; ++k) s += sh[k][q];
        partial[(long)blockIdx.x * BK_MAXM + q] = s;
    }
}

// out[p * ostride + q] (= or +=) the sum of process p's chunk partials, one warp per (p, q).
__global__ void k_bdots_final(const double *__restrict__ partial, const BProc *__restrict__ pr, int P, int nq,
                              double *__restrict__ out, long ostride, int accumulate, const int *__restrict__ act) {
    const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long)P * nq) return;
    const int p = (int)(wid / nq), q = (int)(wid % nq);
    if (!act[p]) return;
    double s = 0.0;
    for (int c = pr[p].c0 + lane; c < pr[p].c1; c += 32) s += partial[(long)c * BK_MAXM + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double *o_ = out + (long)p * ostride + q;
        *o_ = accumulate ? *o_ + s : s;
    }
}

// w(rows, col) -= sum_q V_q(rows, col) h_p[q], q < nq  (h_p = h + p * hstride)
__global__ void k_bsub_Vh(const double *__restrict__ V, long ldv, long vstride, int nq, const double *__restrict__ h,
                          long hstride, double *__restrict__ w, long ldw, const BChunk *__restrict__ ch,
                          const int *__restrict__ act) {
    const BChunk C = ch[blockIdx.x];
    if (!act[C.p]) return;
    __shared__ double hs[BK_MAXM];
    if (threadIdx.x < nq) hs[threadIdx.x] = h[(long)C.p * hstride + threadIdx.x];
    __syncthreads();
    double *wc = w + (long)C.col * ldw + C.row0;
    const double *vc = V + (long)C.col * ldv + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) {
        double acc = wc[i];
        for (int q = 0; q < nq; ++q) acc -= vc[i + vstride * q] * hs[q];
        wc[i] = acc;
    }
}

// y(rows, col) = x(rows, col) / s_p (s_p == 0 gives 0); s_p = s[p * sstride]
__global__ void k_bscale(const double *__restrict__ x, long ldx, const double *__restrict__ s, long sstride,
                         double *__restrict__ y, long ldy, const BChunk *__restrict__ ch, const int *__restrict__ act) {
    const BChunk C = ch[blockIdx.x];
    if (!act[C.p]) return;
    const double d = s[(long)C.p * sstride];
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    const double *xc = x + (long)C.col * ldx + C.row0;
    double *yc = y + (long)C.col * ldy + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) yc[i] = xc[i] * inv;
}

// r(rows, col) = b(rows, col) - r(rows, col)
__global__ void k_bresid(const double *__restrict__ b, long ldb, double *__restrict__ r, long ldr,
                         const BChunk *__restrict__ ch, const int *__restrict__ act) {
    const BChunk C = ch[blockIdx.x];
    if (!act[C.p]) return;
    const double *bc = b + (long)C.col * ldb + C.row0;
    double *rc = r + (long)C.col * ldr + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) rc[i] = bc[i] - rc[i];
}

// x(rows, col) = 0 for the processes whose right-hand side is zero
__global__ void k_bzero(double *__restrict__ x, long ldx, const BChunk *__restrict__ ch, const int *__restrict__ sel) {
    const BChunk C = ch[blockIdx.x];
    if (!sel[C.p]) return;
    double *xc = x + (long)C.col * ldx + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) xc[i] = 0.0;
}

// out[p * so] = sqrt(in[p * si])
__global__ void k_bsqrt(const double *__restrict__ in, long si, double *__restrict__ out, long so, int P,
                        const int *__restrict__ act) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P && act[p]) out[(long)p * so] = sqrt(in[(long)p * si]);
}

// h_p[q] += y_p[q], q < nq (the second Gram-Schmidt pass)
__global__ void k_badd(double *__restrict__ h, long hstride, const double *__restrict__ y, long ystride, int nq,
                       int P, const int *__restrict__ act) {
    const int p = blockIdx.x, q = threadIdx.x;
    if (p < P && q < nq && act[p]) h[(long)p * hstride + q] += y[(long)p * ystride + q];
}

// Hessenberg column j of each active process: earlier rotations, rotation j, g update;
// est[p] = |g_p[j + 1]|.  Per-process state: H (m+1) x m, cs[m], sn[m], g[m+1].
__global__ void k_bgivens(double *__restrict__ H, int m, int j, double *__restrict__ cs, double *__restrict__ sn,
                          double *__restrict__ g, double *__restrict__ est, int P, const int *__restrict__ act) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !act[p]) return;
    double *h = H + (long)p * (m + 1) * m + (long)(m + 1) * j;
    double *c_ = cs + (long)p * m, *s_ = sn + (long)p * m, *gp = g + (long)p * (m + 1);
    for (int i = 0; i < j; ++i) {
        double a = h[i], c = h[i + 1];
        h[i] = c_[i] * a + s_[i] * c;
        h[i + 1] = -s_[i] * a + c_[i] * c;
    }
    double a = h[j], c = h[j + 1];
    double rr = hypot(a, c);
    double cj = rr > 0.0 ? a / rr : 1.0, sj = rr > 0.0 ? c / rr : 0.0;
    c_[j] = cj;
    s_[j] = sj;
    h[j] = rr;
    h[j + 1] = 0.0;
    gp[j + 1] = -sj * gp[j];
    gp[j] = cj * gp[j];
    est[p] = fabs(gp[j + 1]);
}

// g_p = (beta_p, 0, ..., 0)
__global__ void k_binit_g(double *__restrict__ g, int m, const double *__restrict__ beta, long bstride, int P,
                          const int *__restrict__ act) {
    const int p = blockIdx.x;
    if (p >= P || !act[p]) return;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[(long)p * (m + 1) + i] = i == 0 ? beta[(long)p * bstride] : 0.0;
}

// y_p = R_p^-1 g_p on the leading jend_p x jend_p triangle
__global__ void k_bbacksolve(const double *__restrict__ H, int m, const int *__restrict__ jend,
                             const double *__restrict__ g, double *__restrict__ y, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int je = jend[p];
    const double *Hp = H + (long)p * (m + 1) * m;
    const double *gp = g + (long)p * (m + 1);
    double *yp = y + (long)p * m;
    for (int i = je - 1; i >= 0; --i) {
        double s = gp[i];
        for (int l = i + 1; l < je; ++l) s -= Hp[i + (long)(m + 1) * l] * yp[l];
        yp[i] = s / Hp[i + (long)(m + 1) * i];
    }
}

// x(rows, col) += sum_{q < jend_p} Z_q(rows, col) y_p[q]
__global__ void k_bupdate_x(const double *__restrict__ Z, long ldz, long zstride, const int *__restrict__ jend,
                            const double *__restrict__ y, int m, double *__restrict__ x, long ldx,
                            const BChunk *__restrict__ ch) {
    const BChunk C = ch[blockIdx.x];
    const int je = jend[C.p];
    if (je == 0) return;
    __shared__ double ys[BK_MAXM];
    if (threadIdx.x < je) ys[threadIdx.x] = y[(long)C.p * m + threadIdx.x];
    __syncthreads();
    const double *zc = Z + (long)C.col * ldz + C.row0;
    double *xc = x + (long)C.col * ldx + C.row0;
    for (int i = threadIdx.x; i < C.len; i += BK_NT) {
        double acc = xc[i];
        for (int q = 0; q < je; ++q) acc += zc[i + zstride * q] * ys[q];
        xc[i] = acc;
    }
}

}  // namespace
}  // namespace hssnd

using namespace hssnd;

namespace hssnd {

// The lock-step solver: one Krylov process per (instance, right-hand side),
// instance i owning rows [inst_dof[i], inst_dof[i + 1]) of the block vectors.
// A is the (block-diagonal) matrix of all instances, pc its preconditioner
// (HSS, ILU(0) or none), stats one entry per instance, hist (optional) one residual
// history per process.
int fgmres_lockstep(const hss_bsr *A, const Precond &pc, const std::vector<int> &inst_dof, int nrhs,
                    const double *b, int ldb, double *x, int ldx, const fgmres_opts &o, fgmres_stats *stats,
                    std::vector<std::vector<double>> *hist, cudaStream_t s) {
    const int ninst = (int)inst_dof.size() - 1, m = o.restart;
    const long N = inst_dof.back();
    const int P = ninst * nrhs;
    if (stats)
        for (int i = 0; i < ninst; ++i) stats[i] = fgmres_stats{0, 0, 0.0, 1};
    if (hist) hist->assign(P, {});
    if (P == 0 || N == 0) return HSS_OK;

    // processes (column-major over instances) and their row chunks
    std::vector<BProc> pr(P);
    std::vector<BChunk> ch;
    for (int c = 0; c < nrhs; ++c)
        for (int i = 0; i < ninst; ++i) {
            const int p = c * ninst + i;
            const int r0 = inst_dof[i], len = inst_dof[i + 1] - r0;
            pr[p] = BProc{c, r0, len, (int)ch.size(), 0};
            for (int q = 0; q < len; q += BK_CHUNK) ch.push_back(BChunk{p, c, r0 + q, std::min(BK_CHUNK, len - q)});
            pr[p].c1 = (int)ch.size();
        }
    const int nch = (int)ch.size();
    const long NB = N * nrhs;
    DevBuf V, Z, w, r, part, H, cs, sn, g, y, scal, est, act, jend, sel, d_ch, d_pr;
    int rc;
    if ((rc = V.alloc(sizeof(double) * NB * (m + 1))) || (rc = Z.alloc(sizeof(double) * NB * m)) ||
        (rc = w.alloc(sizeof(double) * NB)) || (rc = r.alloc(sizeof(double) * NB)) ||
        (rc = part.alloc(sizeof(double) * (size_t)nch * BK_MAXM)) ||
        (rc = H.alloc(sizeof(double) * (size_t)P * (m + 1) * m)) || (rc = cs.alloc(sizeof(double) * (size_t)P * m)) ||
        (rc = sn.alloc(sizeof(double) * (size_t)P * m)) || (rc = g.alloc(sizeof(double) * (size_t)P * (m + 1))) ||
        (rc = y.alloc(sizeof(double) * (size_t)P * m)) || (rc = scal.alloc(sizeof(double) * (size_t)P * 8)) ||
        (rc = est.alloc(sizeof(double) * P)) || (rc = act.alloc(sizeof(int) * P)) ||
        (rc = jend.alloc(sizeof(int) * P)) || (rc = sel.alloc(sizeof(int) * P)) || (rc = upload(d_ch, ch, s)) ||
        (rc = upload(d_pr, pr, s)))
        return rc;
    double *dV = V.as<double>(), *dZ = Z.as<double>(), *dw = w.as<double>(), *dr = r.as<double>();
    double *dpart = part.as<double>(), *dH = H.as<double>(), *dsc = scal.as<double>();
    const BChunk *dch = d_ch.as<BChunk>();
    const BProc *dpr = d_pr.as<BProc>();
    int *dact = act.as<int>();
    const long hst = (long)(m + 1) * m;

    auto dots = [&](const double *Vb, long ldv, long vstride, int nq, const double *wb, long ldw, double *out,
                    long ostride, int accumulate) -> int {
        { HSS_PROF("bdots", s); k_bdots<<<nch, BK_NT, 0, s>>>(Vb, ldv, vstride, nq, wb, ldw, dch, dact, dpart); }
        {
            HSS_PROF("bdots_final", s);
            const long threads = (long)P * nq * 32;
            k_bdots_final<<<(int)cdiv(threads, 256L), 256, 0, s>>>(dpart, dpr, P, nq, out, ostride, accumulate, dact);
        }
        HSS_CHECK_LAUNCH("batched dots");
        return HSS_OK;
    };
    std::vector<int> act_h(P, 1), done(P, 0), conv(P, 0), iters(P, 0), jend_h(P, 0);
    std::vector<double> bnorm(P, 0.0), relres(P, 0.0), hv((size_t)P * 8), eh(P);
    auto push_act = [&]() -> int {
        HSS_CUDA(cudaMemcpyAsync(dact, act_h.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
        return HSS_OK;
    };
    auto read_scal = [&]() -> int {
        HSS_CUDA(cudaMemcpyAsync(hv.data(), dsc, sizeof(double) * P * 8, cudaMemcpyDeviceToHost, s));
        HSS_CUDA(cudaStreamSynchronize(s));
        return HSS_OK;
    };
    const int pb = cdiv(P, 128);
    // ||b|| per process
    if ((rc = push_act()) || (rc = dots(b, ldb, 0, 1, b, ldb, dsc + 0, 8, 0))) return rc;
    { HSS_PROF("bsqrt", s); k_bsqrt<<<pb, 128, 0, s>>>(dsc + 0, 8, dsc + 1, 8, P, dact); }
    if ((rc = read_scal())) return rc;
    std::vector<int> zero(P, 0);
    bool any_zero = false;
    for (int p = 0; p < P; ++p) {
        bnorm[p] = hv[(size_t)p * 8 + 1];
        if (bnorm[p] == 0.0) {
            zero[p] = 1;
            done[p] = conv[p] = 1;
            any_zero = true;
        }
    }
    if (any_zero) {
        HSS_CUDA(cudaMemcpyAsync(sel.p, zero.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
        { HSS_PROF("bzero", s); k_bzero<<<nch, BK_NT, 0, s>>>(x, ldx, dch, sel.as<int>()); }
        HSS_CHECK_LAUNCH("k_bzero");
    }
    while (true) {
        int nact = 0;
        for (int p = 0; p < P; ++p) nact += (act_h[p] = !done[p]);
        if (nact == 0) break;
        // r = b - A x, beta = ||r||
        if ((rc = push_act()) || (rc = spmv(A, nrhs, x, ldx, dr, N, s))) return rc;
        { HSS_PROF("bresid", s); k_bresid<<<nch, BK_NT, 0, s>>>(b, ldb, dr, N, dch, dact); }
        if ((rc = dots(dr, N, 0, 1, dr, N, dsc + 2, 8, 0))) return rc;
        { HSS_PROF("bsqrt", s); k_bsqrt<<<pb, 128, 0, s>>>(dsc + 2, 8, dsc + 3, 8, P, dact); }
        if ((rc = read_scal())) return rc;
        nact = 0;
        for (int p = 0; p < P; ++p) {
            if (done[p]) continue;
            relres[p] = hv[(size_t)p * 8 + 3] / bnorm[p];
            if (relres[p] <= o.rtol) done[p] = conv[p] = 1;
            else if (iters[p] >= o.maxit || !(relres[p] == relres[p])) done[p] = 1;
            nact += (act_h[p] = !done[p]);
        }
        if (nact == 0) break;
        if ((rc = push_act())) return rc;
        { HSS_PROF("bscale", s); k_bscale<<<nch, BK_NT, 0, s>>>(dr, N, dsc + 3, 8, dV, N, dch, dact); }
        { HSS_PROF("binit_g", s); k_binit_g<<<P, 64, 0, s>>>(g.as<double>(), m, dsc + 3, 8, P, dact); }
        HSS_CUDA(cudaMemsetAsync(dH, 0, sizeof(double) * (size_t)P * hst, s));
        std::fill(jend_h.begin(), jend_h.end(), 0);
        for (int j = 0; j < m; ++j) {
            const double *Vj = dV + NB * j;
            double *Zj = dZ + NB * j;
            if (!pc.none()) {
                if ((rc = precond_apply(pc, nrhs, Vj, N, Zj, N, s))) return rc;
            } else {
                HSS_CUDA(cudaMemcpyAsync(Zj, Vj, sizeof(double) * NB, cudaMemcpyDeviceToDevice, s));
            }
            if ((rc = spmv(A, nrhs, Zj, N, dw, N, s))) return rc;
            double *hcol = dH + (long)(m + 1) * j;
            // classical Gram-Schmidt, twice; the second pass's coefficients are added to the column
            if ((rc = dots(dV, N, NB, j + 1, dw, N, hcol, hst, 0))) return rc;
            { HSS_PROF("bsub_Vh", s); k_bsub_Vh<<<nch, BK_NT, 0, s>>>(dV, N, NB, j + 1, hcol, hst, dw, N, dch, dact); }
            if ((rc = dots(dV, N, NB, j + 1, dw, N, y.as<double>(), m, 0))) return rc;
            { HSS_PROF("bsub_Vh", s); k_bsub_Vh<<<nch, BK_NT, 0, s>>>(dV, N, NB, j + 1, y.as<double>(), m, dw, N, dch, dact); }
            { HSS_PROF("badd", s); k_badd<<<P, 32, 0, s>>>(hcol, hst, y.as<double>(), m, j + 1, P, dact); }
            if ((rc = dots(dw, N, 0, 1, dw, N, dsc + 4, 8, 0))) return rc;
            { HSS_PROF("bsqrt", s); k_bsqrt<<<pb, 128, 0, s>>>(dsc + 4, 8, hcol + j + 1, hst, P, dact); }
            { HSS_PROF("bscale", s); k_bscale<<<nch, BK_NT, 0, s>>>(dw, N, hcol + j + 1, hst, dV + NB * (j + 1), N, dch, dact); }
            { HSS_PROF("bgivens", s); k_bgivens<<<pb, 128, 0, s>>>(dH, m, j, cs.as<double>(), sn.as<double>(), g.as<double>(), est.as<double>(), P, dact); }
            HSS_CHECK_LAUNCH("batched arnoldi step");
            HSS_CUDA(cudaMemcpyAsync(eh.data(), est.p, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
            HSS_CUDA(cudaStreamSynchronize(s));
            bool changed = false;
            nact = 0;
            for (int p = 0; p < P; ++p) {
                if (!act_h[p]) continue;
                ++iters[p];
                jend_h[p] = j + 1;
                const double e = eh[p] / bnorm[p];
                if (hist) (*hist)[p].push_back(e);
                if (e <= o.rtol || iters[p] >= o.maxit || !(e == e)) {
                    act_h[p] = 0;
                    changed = true;
                }
                nact += act_h[p];
            }
            if (nact == 0) break;
            if (changed && (rc = push_act())) return rc;
        }
        HSS_CUDA(cudaMemcpyAsync(jend.p, jend_h.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
        { HSS_PROF("bbacksolve", s); k_bbacksolve<<<pb, 128, 0, s>>>(dH, m, jend.as<int>(), g.as<double>(), y.as<double>(), P); }
        { HSS_PROF("bupdate_x", s); k_bupdate_x<<<nch, BK_NT, 0, s>>>(dZ, N, NB, jend.as<int>(), y.as<double>(), m, x, ldx, dch); }
        HSS_CHECK_LAUNCH("batched fgmres update");
    }
    HSS_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int p = 0; p < P; ++p) {
        const int i = p % ninst;
        if (stats) {
            stats[i].iters += iters[p];
            stats[i].max_iters = std::max(stats[i].max_iters, iters[p]);
            stats[i].relres = std::max(stats[i].relres, relres[p]);
            if (!conv[p]) stats[i].converged = 0;
        }
        all = all && conv[p];
    }
    return all ? HSS_OK : HSS_ENOCONV;
}

}  // namespace hssnd

extern "C" int fgmres_solve_batched(const hss_factor_t *f, int nrhs, const double *b, int ldb, double *x, int ldx,
                                    const fgmres_opts *opts, fgmres_stats *stats, void *stream) {
    fgmres_opts o;
    fgmres_opts_default(&o);
    if (opts) o = *opts;
    const long N = f ? f->ndof : 0;
    if (!f || !f->batched || !b || !x || nrhs < 0 || ldb < N || ldx < N || o.restart < 1 ||
        o.restart > BK_MAXM - 1 || o.maxit < 0) {
        set_error("fgmres_solve_batched: invalid argument (needs a factor from hss_factor_batched; restart in [1, 31])");
        return HSS_EINVAL;
    }
    return fgmres_lockstep(&f->bA, Precond{f, nullptr}, f->tree->inst_dof, nrhs, b, ldb, x, ldx, o, stats, nullptr,
                           (cudaStream_t)stream);
}
