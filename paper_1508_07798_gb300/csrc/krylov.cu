// Block-sparse SpMV and right-preconditioned restarted flexible GMRES.
//
// The paper measures its preconditioner by GMRES iterations (Sec. 5).  Each
// Arnoldi step here: z_j = M^-1 v_j (hss_apply), w = A z_j (SpMV), classical
// Gram-Schmidt applied twice against V (two reductions + updates each), the
// new basis vector, and one Givens rotation of the Hessenberg column, all on
// the device.  The host reads one residual estimate per step to stop.
#include <cmath>

#include "factor.h"
#include "prof.h"

namespace hssnd {

constexpr int KRY_NT = 256;
constexpr int KRY_MAXM = 32;      // largest restart length + 1
constexpr int DOT_BLOCKS = 304;   // 2 x 152 SMs

// y = A x, one thread per scalar row and right-hand side.
__global__ void k_spmv(int nb, int bs, const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                       const double *__restrict__ val, const double *__restrict__ x, long ldx,
                       double *__restrict__ y, long ldy, int nrhs) {
    pdl_launch_next();
    pdl_wait_prev();
    long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long N = (long)nb * bs;
    if (g >= N * nrhs) return;
    int rr = (int)(g / N);
    int row = (int)(g % N);
    int e = row / bs, r = row % bs;
    const double *xv = x + ldx * rr;
    double acc = 0.0;
    for (int t = row_ptr[e]; t < row_ptr[e + 1]; ++t) {
        const double *blk = val + ((long)t * bs + r) * bs;
        const double *xs = xv + (long)col_idx[t] * bs;
        for (int c = 0; c < bs; ++c) acc = fma(blk[c], xs[c], acc);
    }
    y[row + ldy * rr] = acc;
}

// y = A x for several right-hand sides: one thread per scalar row, the row's
// blocks read once for up to SPMV_RB right-hand sides (same summation order
// per right-hand side as k_spmv).
constexpr int SPMV_RB = 8;
__global__ void k_spmv_multi(int nb, int bs, const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                             const double *__restrict__ val, const double *__restrict__ x, long ldx,
                             double *__restrict__ y, long ldy, int nrhs) {
    pdl_launch_next();
    pdl_wait_prev();
    long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long N = (long)nb * bs;
    if (row >= N) return;
    int e = (int)(row / bs), r = (int)(row % bs);
    for (int r0 = 0; r0 < nrhs; r0 += SPMV_RB) {
        const int nr = min(SPMV_RB, nrhs - r0);
        double acc[SPMV_RB];
#pragma unroll
        for (int k = 0; k < SPMV_RB; ++k) acc[k] = 0.0;
        for (int t = row_ptr[e]; t < row_ptr[e + 1]; ++t) {
            const double *blk = val + ((long)t * bs + r) * bs;
            const double *xs = x + (long)col_idx[t] * bs + ldx * r0;
            for (int c = 0; c < bs; ++c) {
                const double a = blk[c];
#pragma unroll
                for (int k = 0; k < SPMV_RB; ++k)
                    if (k < nr) acc[k] = fma(a, xs[c + ldx * k], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < SPMV_RB; ++k)
            if (k < nr) y[row + ldy * (r0 + k)] = acc[k];
    }
}

// partial[b * KRY_MAXM + q] = sum over this CTA's rows of V(:,q) . w, q < nq
__global__ void k_dots(const double *__restrict__ V, long ldv, int nq, const double *__restrict__ w, long N,
                       double *__restrict__ partial) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ double sh[KRY_NT / 32][KRY_MAXM + 1];
    double acc[KRY_MAXM];
#pragma unroll
    for (int q = 0; q < KRY_MAXM; ++q) acc[q] = 0.0;
    for (long i = (long)blockIdx.x * KRY_NT + threadIdx.x; i < N; i += (long)gridDim.x * KRY_NT) {
        double wi = w[i];
#pragma unroll
        for (int q = 0; q < KRY_MAXM; ++q)
            if (q < nq) acc[q] = fma(V[i + ldv * q], wi, acc[q]);
    }
    int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < KRY_MAXM; ++q) {
        if (q >= nq) break;
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += KRY_NT) {
        double s = 0.0;
        for (int k = 0; k < KRY_NT / 32; ++k) s += sh[k][q];
        partial[(long)blockIdx.x * KRY_MAXM + q] = s;
    }
}

// out[q] (= or +=) sum of the partials, q < nq, one warp per q, fixed order.
__global__ void k_dots_final(const double *__restrict__ partial, int nblk, int nq, double *__restrict__ out,
                             int accumulate) {
    pdl_launch_next();
    pdl_wait_prev();
    int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[(long)b * KRY_MAXM + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[q] = accumulate ? out[q] + s : s;
}

// w -= V(:, 0:nq) h
__global__ void k_sub_Vh(const double *__restrict__ V, long ldv, int nq, const double *__restrict__ h,
                         double *__restrict__ w, long N) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ double hs[KRY_MAXM];
    if (threadIdx.x < nq) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (long i = (long)blockIdx.x * KRY_NT + threadIdx.x; i < N; i += (long)gridDim.x * KRY_NT) {
        double acc = w[i];
        for (int q = 0; q < nq; ++q) acc -= V[i + ldv * q] * hs[q];
        w[i] = acc;
    }
}

// y = alpha * x / s[0] (s on the device; s[0] == 0 leaves y = 0)
__global__ void k_scale_by(const double *__restrict__ x, const double *__restrict__ s, double *__restrict__ y,
                           long N) {
    pdl_launch_next();
    pdl_wait_prev();
    double d = s[0];
    double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (long i = (long)blockIdx.x * KRY_NT + threadIdx.x; i < N; i += (long)gridDim.x * KRY_NT) y[i] = x[i] * inv;
}

__global__ void k_sqrt_into(const double *__restrict__ s2, double *__restrict__ out) {
    pdl_launch_next();
    pdl_wait_prev();
    if (threadIdx.x == 0) out[0] = sqrt(s2[0]);
}

// r = b - r (r holds A x)
__global__ void k_resid(const double *__restrict__ b, double *__restrict__ r, long N) {
    pdl_launch_next();
    pdl_wait_prev();
    for (long i = (long)blockIdx.x * KRY_NT + threadIdx.x; i < N; i += (long)gridDim.x * KRY_NT) r[i] = b[i] - r[i];
}

// Hessenberg column j: apply the earlier rotations, form rotation j, update g.
// State layout: H (m+1) x m column-major, cs[m], sn[m], g[m+1]; est = |g[j+1]|.
__global__ void k_givens(double *__restrict__ H, int m, int j, double *__restrict__ cs, double *__restrict__ sn,
                         double *__restrict__ g, double *__restrict__ est) {
    pdl_launch_next();
    pdl_wait_prev();
    if (threadIdx.x != 0) return;
    double *h = H + (long)(m + 1) * j;
    for (int i = 0; i < j; ++i) {
        double a = h[i], c = h[i + 1];
        h[i] = cs[i] * a + sn[i] * c;
        h[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = h[j], c = h[j + 1];
    double rr = hypot(a, c);
    double cj = rr > 0.0 ? a / rr : 1.0, sj = rr > 0.0 ? c / rr : 0.0;
    cs[j] = cj;
    sn[j] = sj;
    h[j] = rr;
    h[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
    est[0] = fabs(g[j + 1]);
}

// y = R^-1 g for the leading jend x jend triangle of H
__global__ void k_backsolve(const double *__restrict__ H, int m, int jend, const double *__restrict__ g,
                            double *__restrict__ y) {
    pdl_launch_next();
    pdl_wait_prev();
    if (threadIdx.x != 0) return;
    for (int i = jend - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < jend; ++l) s -= H[i + (long)(m + 1) * l] * y[l];
        y[i] = s / H[i + (long)(m + 1) * i];
    }
}

// x += Z(:, 0:jend) y
__global__ void k_update_x(const double *__restrict__ Z, long ldz, int jend, const double *__restrict__ y,
                           double *__restrict__ x, long N) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ double ys[KRY_MAXM];
    if (threadIdx.x < jend) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (long i = (long)blockIdx.x * KRY_NT + threadIdx.x; i < N; i += (long)gridDim.x * KRY_NT) {
        double acc = x[i];
        for (int q = 0; q < jend; ++q) acc += Z[i + ldz * q] * ys[q];
        x[i] = acc;
    }
}

__global__ void k_init_g(double *__restrict__ g, int m, const double *__restrict__ beta) {
    pdl_launch_next();
    pdl_wait_prev();
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? beta[0] : 0.0;
}

static double spmv_bytes(const hss_bsr *A, int nrhs) {
    // block values and column indices once, row pointers, x read and y written per right-hand side;
    // computed only while profiling, the block count cached per matrix
    if (!prof_enabled()) return 0.0;
    static const int *cached_ptr = nullptr;
    static int cached_nnzb = 0;
    if (cached_ptr != A->row_ptr) {
        cudaMemcpy(&cached_nnzb, A->row_ptr + A->nb, sizeof(int), cudaMemcpyDeviceToHost);
        cached_ptr = A->row_ptr;
    }
    int nnzb = cached_nnzb;
    double N = (double)A->nb * A->bs;
    return (double)nnzb * A->bs * A->bs * 8.0 + nnzb * 4.0 + (A->nb + 1) * 4.0 + 2.0 * N * 8.0 * nrhs;
}

int spmv(const hss_bsr *A, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s) {
    long N = (long)A->nb * A->bs;
    long tot = N * nrhs;
    if (tot == 0) return HSS_OK;
    if (nrhs == 1) {
        HSS_PROF("spmv", s, spmv_bytes(A, nrhs));
        HSS_CUDA(launch_pdl(k_spmv, dim3(cdiv(tot, KRY_NT)), dim3(KRY_NT), 0, s, A->nb, A->bs, A->row_ptr, A->col_idx, A->val, x, ldx, y, ldy, nrhs));
    } else {
        HSS_PROF("spmv", s, spmv_bytes(A, nrhs));
        HSS_CUDA(launch_pdl(k_spmv_multi, dim3(cdiv(N, KRY_NT)), dim3(KRY_NT), 0, s, A->nb, A->bs, A->row_ptr, A->col_idx, A->val, x, ldx, y, ldy,
                                                       nrhs));
    }
    HSS_CHECK_LAUNCH("k_spmv");
    return HSS_OK;
}

// Krylov workspace of one solve, carved from the call scratch (cached between calls).
struct Krylov {
    ScratchPtr V, Z, w, r, part, H, cs, sn, g, y, scal;
    int m = 0;
    long N = 0;
    int alloc(Work &W, long n, int mm) {
        int rc;
        if ((rc = W.dalloc_bytes(sizeof(double) * n * (mm + 1), &V.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * n * mm, &Z.p)) || (rc = W.dalloc_bytes(sizeof(double) * n, &w.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * n, &r.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * DOT_BLOCKS * KRY_MAXM, &part.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * (mm + 1) * mm, &H.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * mm, &cs.p)) || (rc = W.dalloc_bytes(sizeof(double) * mm, &sn.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * (mm + 1), &g.p)) || (rc = W.dalloc_bytes(sizeof(double) * mm, &y.p)) ||
            (rc = W.dalloc_bytes(sizeof(double) * 8, &scal.p)))
            return rc;
        m = mm;
        N = n;
        return HSS_OK;
    }
};

static thread_local std::vector<std::vector<double>> g_hist;

// sum_i v_i w_i into out[0] (deterministic two-pass)
static int dot1(const double *v, const double *w, long N, double *part, double *out, int acc, cudaStream_t s) {
    { HSS_PROF("dots", s); HSS_CUDA(launch_pdl(k_dots, dim3(DOT_BLOCKS), dim3(KRY_NT), 0, s, v, N, 1, w, N, part)); }
    { HSS_PROF("dots_final", s); HSS_CUDA(launch_pdl(k_dots_final, dim3(1), dim3(32), 0, s, part, DOT_BLOCKS, 1, out, acc)); }
    HSS_CHECK_LAUNCH("dot");
    return HSS_OK;
}

static int fgmres_one(const hss_bsr *A, const Precond &pc, const double *b, double *x, const fgmres_opts &o,
                      Krylov &K, int &iters, double &relres, bool &conv, std::vector<double> &hist, cudaStream_t s) {
    const long N = K.N;
    const int m = K.m;
    double *V = K.V.as<double>(), *Z = K.Z.as<double>(), *w = K.w.as<double>(), *r = K.r.as<double>();
    double *part = K.part.as<double>(), *H = K.H.as<double>(), *sc = K.scal.as<double>();
    const int gb = DOT_BLOCKS;
    int rc;
    double host[2];
    // ||b||
    if ((rc = dot1(b, b, N, part, sc + 0, 0, s))) return rc;
    { HSS_PROF("sqrt_into", s); HSS_CUDA(launch_pdl(k_sqrt_into, dim3(1), dim3(32), 0, s, sc + 0, sc + 1)); }
    HSS_CUDA(cudaMemcpyAsync(host, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    const double bnorm = host[0];
    iters = 0;
    conv = false;
    if (bnorm == 0.0) {
        HSS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
        relres = 0.0;
        conv = true;
        return HSS_OK;
    }
    while (true) {
        // r = b - A x, beta = ||r||
        if ((rc = spmv(A, 1, x, N, r, N, s))) return rc;
        { HSS_PROF("resid", s); HSS_CUDA(launch_pdl(k_resid, dim3(gb), dim3(KRY_NT), 0, s, b, r, N)); }
        if ((rc = dot1(r, r, N, part, sc + 2, 0, s))) return rc;
        { HSS_PROF("sqrt_into", s); HSS_CUDA(launch_pdl(k_sqrt_into, dim3(1), dim3(32), 0, s, sc + 2, sc + 3)); }
        HSS_CUDA(cudaMemcpyAsync(host, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
        HSS_CUDA(cudaStreamSynchronize(s));
        double beta = host[0];
        relres = beta / bnorm;
        if (relres <= o.rtol) {
            conv = true;
            return HSS_OK;
        }
        if (iters >= o.maxit) return HSS_OK;
        { HSS_PROF("scale_by", s); HSS_CUDA(launch_pdl(k_scale_by, dim3(gb), dim3(KRY_NT), 0, s, r, sc + 3, V, N)); }
        { HSS_PROF("init_g", s); HSS_CUDA(launch_pdl(k_init_g, dim3(1), dim3(64), 0, s, K.g.as<double>(), m, sc + 3)); }
        HSS_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * (m + 1) * m, s));
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = V + N * j, *zj = Z + N * j;
            if (!pc.none()) {
                if ((rc = precond_apply(pc, 1, vj, N, zj, N, s))) return rc;
            } else {
                HSS_CUDA(cudaMemcpyAsync(zj, vj, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            }
            if ((rc = spmv(A, 1, zj, N, w, N, s))) return rc;
            double *hcol = H + (long)(m + 1) * j;
            // classical Gram-Schmidt, twice
            for (int pass = 0; pass < 2; ++pass) {
                { HSS_PROF("dots", s); HSS_CUDA(launch_pdl(k_dots, dim3(gb), dim3(KRY_NT), 0, s, V, N, j + 1, w, N, part)); }
                { HSS_PROF("dots_final", s); HSS_CUDA(launch_pdl(k_dots_final, dim3(1), dim3(32 * (j + 1)), 0, s, part, gb, j + 1, pass ? K.y.as<double>() : hcol, 0)); }
                { HSS_PROF("sub_Vh", s); HSS_CUDA(launch_pdl(k_sub_Vh, dim3(gb), dim3(KRY_NT), 0, s, V, N, j + 1, pass ? K.y.as<double>() : hcol, w, N)); }
            }
            // h += h2 (the second-pass coefficients, read as a one-block partial sum)
            { HSS_PROF("dots_final", s); HSS_CUDA(launch_pdl(k_dots_final, dim3(1), dim3(32 * (j + 1)), 0, s, K.y.as<double>(), 1, j + 1, hcol, 1)); }
            if ((rc = dot1(w, w, N, part, sc + 4, 0, s))) return rc;
            { HSS_PROF("sqrt_into", s); HSS_CUDA(launch_pdl(k_sqrt_into, dim3(1), dim3(32), 0, s, sc + 4, hcol + j + 1)); }
            { HSS_PROF("scale_by", s); HSS_CUDA(launch_pdl(k_scale_by, dim3(gb), dim3(KRY_NT), 0, s, w, hcol + j + 1, V + N * (j + 1), N)); }
            { HSS_PROF("givens", s); HSS_CUDA(launch_pdl(k_givens, dim3(1), dim3(32), 0, s, H, m, j, K.cs.as<double>(), K.sn.as<double>(), K.g.as<double>(), sc + 5)); }
            HSS_CHECK_LAUNCH("arnoldi step");
            HSS_CUDA(cudaMemcpyAsync(host, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
            HSS_CUDA(cudaStreamSynchronize(s));
            ++iters;
            jend = j + 1;
            double est = host[0] / bnorm;
            hist.push_back(est);
            if (est <= o.rtol || iters >= o.maxit || !(est == est)) break;
        }
        { HSS_PROF("backsolve", s); HSS_CUDA(launch_pdl(k_backsolve, dim3(1), dim3(32), 0, s, H, m, jend, K.g.as<double>(), K.y.as<double>())); }
        { HSS_PROF("update_x", s); HSS_CUDA(launch_pdl(k_update_x, dim3(gb), dim3(KRY_NT), 0, s, Z, N, jend, K.y.as<double>(), x, N)); }
        HSS_CHECK_LAUNCH("fgmres update");
    }
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_spmv(const hss_bsr *A, int nrhs, const double *x, int ldx, double *y, int ldy, void *stream) {
    if (!A || !x || !y || nrhs < 0 || ldx < A->nb * A->bs || ldy < A->nb * A->bs) {
        set_error("hss_spmv: invalid argument");
        return HSS_EINVAL;
    }
    return spmv(A, nrhs, x, ldx, y, ldy, (cudaStream_t)stream);
}

// fgmres_solve for any right preconditioner: one Krylov space at a time for a
// single right-hand side, lock-step processes for several.
static int fgmres_driver(const hss_bsr *A, const Precond &pc, int nrhs, const double *b, int ldb, double *x, int ldx,
                         const fgmres_opts &o, fgmres_stats *stats, cudaStream_t s) {
    const long N = (long)A->nb * A->bs;
    if (nrhs > 1) {
        // several right-hand sides: independent Krylov processes in lock step,
        // one multi-vector apply and SpMV per Arnoldi step
        fgmres_stats st{0, 0, 0.0, 1};
        int rc = fgmres_lockstep(A, pc, std::vector<int>{0, (int)N}, nrhs, b, ldb, x, ldx, o, &st, &g_hist, s);
        if (rc != HSS_OK && rc != HSS_ENOCONV) return rc;
        if (stats) *stats = st;
        return st.converged ? HSS_OK : HSS_ENOCONV;
    }
    Work W(s);
    Krylov K;
    int rc;
    if ((rc = K.alloc(W, N, o.restart))) return rc;
    g_hist.assign(nrhs, {});
    fgmres_stats st{0, 0, 0.0, 1};
    for (int k = 0; k < nrhs; ++k) {
        int it = 0;
        double rel = 0;
        bool conv = false;
        if ((rc = fgmres_one(A, pc, b + (long)ldb * k, x + (long)ldx * k, o, K, it, rel, conv, g_hist[k], s)))
            return rc;
        st.iters += it;
        st.max_iters = std::max(st.max_iters, it);
        st.relres = std::max(st.relres, rel);
        if (!conv) st.converged = 0;
    }
    if (stats) *stats = st;
    return st.converged ? HSS_OK : HSS_ENOCONV;
}

static bool fgmres_args_ok(const hss_bsr *A, int nrhs, const double *b, int ldb, const double *x, int ldx,
                           const fgmres_opts &o, long M_ndof) {
    const long N = A ? (long)A->nb * A->bs : 0;
    return A && b && x && nrhs >= 0 && ldb >= N && ldx >= N && o.restart >= 1 && o.restart <= KRY_MAXM - 1 &&
           o.maxit >= 0 && (M_ndof < 0 || M_ndof == N);
}

extern "C" int fgmres_solve(const hss_bsr *A, const hss_factor_t *f, int nrhs, const double *b, int ldb, double *x,
                            int ldx, const fgmres_opts *opts, fgmres_stats *stats, void *stream) {
    fgmres_opts o;
    fgmres_opts_default(&o);
    if (opts) o = *opts;
    if (!fgmres_args_ok(A, nrhs, b, ldb, x, ldx, o, f ? (long)f->ndof : -1)) {
        set_error("fgmres_solve: invalid argument (restart must be in [1, 31])");
        return HSS_EINVAL;
    }
    return fgmres_driver(A, Precond{f, nullptr}, nrhs, b, ldb, x, ldx, o, stats, (cudaStream_t)stream);
}

extern "C" int fgmres_solve_ilu0(const hss_bsr *A, const hss_ilu_t *M, int nrhs, const double *b, int ldb,
                                 double *x, int ldx, const fgmres_opts *opts, fgmres_stats *stats, void *stream) {
    fgmres_opts o;
    fgmres_opts_default(&o);
    if (opts) o = *opts;
    if (!M || !fgmres_args_ok(A, nrhs, b, ldb, x, ldx, o, ilu_ndof(M))) {
        set_error("fgmres_solve_ilu0: invalid argument (null preconditioner, size mismatch, or restart outside [1, 31])");
        return HSS_EINVAL;
    }
    return fgmres_driver(A, Precond{nullptr, M}, nrhs, b, ldb, x, ldx, o, stats, (cudaStream_t)stream);
}

extern "C" int fgmres_history(int rhs, double *hist, int cap) {
    if (rhs < 0 || rhs >= (int)g_hist.size()) return 0;
    int n = std::min<int>(cap, (int)g_hist[rhs].size());
    for (int i = 0; i < n; ++i) hist[i] = g_hist[rhs][i];
    return n;
}
