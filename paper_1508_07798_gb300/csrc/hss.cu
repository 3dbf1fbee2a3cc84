// Randomized HSS construction of a Schur complement (paper Sec. 2, Theorem 1)
// with interpolative decompositions (Sec. 2, eq. (43) and its footnote).
//
// Per HSS node and side (rows: U, J; columns: V, K), one CTA:
//   local samples  leaf:   Y(R,:) - S(R,R) Omega(R,:)           (precomputed by GEMM)
//                  parent: [Y_a(J_a,:) - S(J_a,K_b) Om_b ; Y_b(J_b,:) - S(J_b,K_a) Om_a]
//                  (columns: Z with S^t and Psi)
//   row ID         column-pivoted Householder QR of the transposed samples,
//                  rank k = first j with |R_jj| <= tol |R_11|, T = R11^-1 R12,
//                  exchanges while some |T_ij| > 2 (largest entry first)
//   outputs        k, skeleton indices, T, skeleton samples, and the
//                  compressed test matrix U^t Psi_loc (rows) / V^t Omega_loc (cols)
// Then, bottom-up, the tall bases U^tall = diag(U^tall_a, U^tall_b) U, and the
// dense approximant H = D on leaf blocks, U^tall_a S(J_a,K_b) V^tall_b^t across
// siblings, written straight into the parent front (eq. (32)).
#include <climits>
#include <type_traits>

#include "hss.h"
#include "prof.h"

namespace hssnd {

// Argmax over non-negative values by their IEEE bit patterns (monotonic for
// v >= 0; -1 = no candidate): integer compares only.
template <class T> struct AM {
    long long v;
    int i;
};
__device__ __forceinline__ long long nn_key(float a) { return (long long)(unsigned)__float_as_int(a); }
__device__ __forceinline__ long long nn_key(double a) { return __double_as_longlong(a); }
__device__ __forceinline__ long long abs_key(float a) { return (long long)(__float_as_int(a) & 0x7fffffff); }
__device__ __forceinline__ long long abs_key(double a) { return __double_as_longlong(a) & 0x7fffffffffffffffLL; }
__device__ __forceinline__ float key_val(long long k, float) { return __int_as_float((int)k); }
__device__ __forceinline__ double key_val(long long k, double) { return __longlong_as_double(k); }

// FP32 keys (non-negative IEEE bit patterns, -1 = none) fit in 31 bits: the
// warp argmax is two reductions, the largest key + 1, then the lowest index
// holding it (ties to the lowest index, as in the shuffle form).
__device__ __forceinline__ AM<float> warp_am_redux(AM<float> x) {
    const unsigned k = (unsigned)(x.v + 1);
    const unsigned m = __reduce_max_sync(0xffffffffu, k);
    const int i = __reduce_min_sync(0xffffffffu, k == m ? x.i : INT_MAX);
    return AM<float>{(long long)m - 1, i};
}

// Argmax of the per-warp candidates (ID_NT / 32 of them), computed by every thread.
template <class T> __device__ __forceinline__ AM<T> reduce_candidates(const AM<T> *c) {
    if constexpr (std::is_same<T, float>::value) {
        const int lane = threadIdx.x & 31;
        return warp_am_redux(lane < ID_NT / 32 ? c[lane] : AM<float>{-1LL, INT_MAX});
    } else {
        AM<T> b = c[0];
        for (int k = 1; k < ID_NT / 32; ++k)
            if (c[k].v > b.v || (c[k].v == b.v && c[k].i < b.i)) b = c[k];
        return b;
    }
}

template <class T> __device__ AM<T> blk_argmax(AM<T> x, AM<T> *sh) {
    if constexpr (std::is_same<T, float>::value) {
        x = warp_am_redux(x);
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            long long v2 = __shfl_down_sync(0xffffffffu, x.v, o);
            int i2 = __shfl_down_sync(0xffffffffu, x.i, o);
            if (v2 > x.v || (v2 == x.v && i2 < x.i)) {
                x.v = v2;
                x.i = i2;
            }
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // previous readers of sh are done
    if (lane == 0) sh[w] = x;
    __syncthreads();
    return reduce_candidates(sh);
}

// 16 bytes of a shared-memory column (4 floats or 2 doubles), 16-byte aligned.
template <class T> __device__ __forceinline__ void ld16(const T *p, T *a) {
    if constexpr (std::is_same<T, float>::value) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a[0] = v.x;
        a[1] = v.y;
        a[2] = v.z;
        a[3] = v.w;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        a[0] = v.x;
        a[1] = v.y;
    }
}
template <class T> __device__ __forceinline__ void st16(T *p, const T *a) {
    if constexpr (std::is_same<T, float>::value)
        *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
    else
        *reinterpret_cast<double2 *>(p) = make_double2(a[0], a[1]);
}

template <class T> __device__ T blk_sum(T x, T *sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        T s = 0;
        for (int k = 0; k < ID_NT / 32; ++k) s += sh[k];
        sh[0] = s;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// Householder step j on A (r x m, leading dimension lda), columns >= j.
template <class T> __device__ void householder_step(T *A, int r, int lda, int m, int j, T nrm, T *v, T *shs) {
    T x0 = A[j + (long)lda * j];
    T alpha = (x0 != T(0)) ? -copysign(nrm, x0) : -nrm;
    for (int i = j + threadIdx.x; i < r; i += ID_NT) v[i] = (i == j) ? x0 - alpha : A[i + (long)lda * j];
    __syncthreads();
    T part = 0;
    for (int i = j + threadIdx.x; i < r; i += ID_NT) part += v[i] * v[i];
    T vn = blk_sum(part, shs);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (vn > T(0)) {
        for (int c = j + 1 + w; c < m; c += ID_NT / 32) {
            T d = 0;
            for (int i = j + lane; i < r; i += 32) d += v[i] * A[i + (long)lda * c];
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            T coef = T(2) * d / vn;
            for (int i = j + lane; i < r; i += 32) A[i + (long)lda * c] -= coef * v[i];
        }
    }
    __syncthreads();
    for (int i = j + threadIdx.x; i < r; i += ID_NT) A[i + (long)lda * j] = (i == j) ? alpha : T(0);
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(ID_NT) k_hss_id(const NodeDev *__restrict__ nodes, const int *__restrict__ work,
                                                const CompFront<T> *__restrict__ cfs, T *__restrict__ ws,
                                                int *__restrict__ iws, int *__restrict__ kout,
                                                int *__restrict__ front_kmax, T tol, uint64_t seed) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ AM<T> sham[ID_NT / 32];
    __shared__ T shs[ID_NT / 32];
    const int node = work[blockIdx.x] >> 1, side = work[blockIdx.x] & 1;
    const NodeDev N = nodes[node];
    const CompFront<T> C = cfs[N.cf];
    const NodeSide me = N.s[side];
    const int r = C.r, mcap = me.mcap, kcap = me.kcap;
    const bool leaf = N.a < 0;
    int ka = 0, m;
    if (leaf) {
        m = N.hi - N.lo;
    } else {
        ka = kout[2 * N.a + side];
        m = ka + kout[2 * N.b + side];
    }
    const int lda = id_lda(r, (int)sizeof(T));           // 16-byte column starts (hss.h)
    T *A = reinterpret_cast<T *>(smraw);                 // r x m, ld lda
    T *v = A + (long)lda * mcap;                          // r
    T *nrm2 = v + r;                                      // mcap
    int *order = reinterpret_cast<int *>(nrm2 + mcap);    // mcap
    T *L = ws + me.loff;                                  // m x r, ld mcap
    const T *S = C.S;
    const long lds = C.lds;

    // ---- local samples
    if (leaf) {
        const T *Ysrc = ws + (side == 0 ? C.yoff : C.zoff);
        for (int idx = threadIdx.x; idx < m * r; idx += ID_NT) {
            int i = idx % m, j = idx / m;
            L[i + (long)mcap * j] = Ysrc[(N.lo + i) + (long)C.nb * j];
        }
        __syncthreads();   // L is read below under a different thread mapping
    } else {
        // coupling blocks staged in shared memory (A's space is free until the QR):
        //   rows: S(J_a, K_b) and S(J_b, K_a); columns: S(J_b, K_a)^t and S(J_a, K_b)^t
        const NodeSide ca = nodes[N.a].s[side], cb = nodes[N.b].s[side];
        const NodeSide oa = nodes[N.a].s[1 - side], ob = nodes[N.b].s[1 - side];
        const int kb_ = m - ka;
        const int koa = kout[2 * N.a + (1 - side)], kob = kout[2 * N.b + (1 - side)];
        T *Ba = A;                       // ka x kob (ld ka)
        T *Bb = A + (long)ka * kob;      // kb x koa (ld kb)
        for (int idx = threadIdx.x; idx < ka * kob; idx += ID_NT) {
            int i = idx % ka, q = idx / ka;
            int gi = iws[ca.skioff + i], go = iws[ob.skioff + q];
            Ba[idx] = side == 0 ? S[gi + lds * go] : S[go + lds * gi];
        }
        for (int idx = threadIdx.x; idx < kb_ * koa; idx += ID_NT) {
            int i = idx % kb_, q = idx / kb_;
            int gi = iws[cb.skioff + i], go = iws[oa.skioff + q];
            Bb[idx] = side == 0 ? S[gi + lds * go] : S[go + lds * gi];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < m * r; idx += ID_NT) {
            int i = idx % m, j = idx / m;
            T val;
            if (i < ka) {
                val = ws[ca.skoff + i + (long)ca.kcap * j];
                const T *tl = ws + ob.tloff + (long)ob.kcap * j;
                for (int q = 0; q < kob; ++q) val -= Ba[i + ka * q] * tl[q];
            } else {
                int ii = i - ka;
                val = ws[cb.skoff + ii + (long)cb.kcap * j];
                const T *tl = ws + oa.tloff + (long)oa.kcap * j;
                for (int q = 0; q < koa; ++q) val -= Bb[ii + kb_ * q] * tl[q];
            }
            L[i + (long)mcap * j] = val;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < m * r; idx += ID_NT) {
        int j = idx % r, i = idx / r;
        A[j + (long)lda * i] = L[i + (long)mcap * j];
    }
    for (int c = threadIdx.x; c < m; c += ID_NT) order[c] = c;
    __syncthreads();

    // ---- column-pivoted QR of A = L^t with the relative rank cut.  One thread
    // per column (c = threadIdx.x + ID_NT q): it applies the step's reflector
    // to its columns in 16-byte pieces, reading the pivot column by broadcast,
    // recomputes their trailing squared norms and offers the largest (ties:
    // lowest column) as its pivot candidate.  Per step, one barrier publishes
    // the candidates and one the interchanged pivot column.  The reflector is
    // v = A(j:r, j) with v_j = x0 - alpha; R(j, j) = alpha is kept in v[j] and
    // placed after the loop (the pivot column is read unchanged during its step).
    constexpr int VW = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ AM<T> cand[ID_NT / 32];
    auto offer = [&](AM<T> mine) {
        if constexpr (std::is_same<T, float>::value) {
            mine = warp_am_redux(mine);
        } else {
            for (int o = 16; o > 0; o >>= 1) {
                const long long v2 = __shfl_xor_sync(0xffffffffu, mine.v, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, mine.i, o);
                if (v2 > mine.v || (v2 == mine.v && i2 < mine.i)) {
                    mine.v = v2;
                    mine.i = i2;
                }
            }
        }
        if (lane == 0) cand[w] = mine;
    };
    {
        AM<T> mine{-1LL, INT_MAX};
        for (int c = threadIdx.x; c < m; c += ID_NT) {
            const T *Ac = A + (long)lda * c;
            T sp[VW] = {};
            for (int q0 = 0; q0 < r; q0 += VW) {
                T a[VW];
                ld16(Ac + q0, a);
#pragma unroll
                for (int e = 0; e < VW; ++e)
                    if (q0 + e < r) sp[e] += a[e] * a[e];
            }
            T sq = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) sq += sp[e];
            const long long kc = nn_key(sq);
            if (kc > mine.v || (kc == mine.v && c < mine.i)) mine = AM<T>{kc, c};
        }
        offer(mine);
    }
    int k = 0;
    T first = 0;
    const int kmx = min(r, m);
    for (int j = 0; j < kmx; ++j) {
        __syncthreads();   // candidates and the updated columns are visible
        const AM<T> best = reduce_candidates(cand);
        const T nn2 = key_val(best.v, T(0));
        const T nrm = sqrt(nn2);
        if (j == 0) first = nrm;
        if (best.v < 0 || first == T(0) || nrm <= tol * first) break;
        const int p = best.i;
        if (p != j) {
            if (threadIdx.x == 0) {
                const int t = order[j];
                order[j] = order[p];
                order[p] = t;
            }
            for (int i = threadIdx.x; i < r; i += ID_NT) {
                const T t = A[i + (long)lda * j];
                A[i + (long)lda * j] = A[i + (long)lda * p];
                A[i + (long)lda * p] = t;
            }
        }
        __syncthreads();   // every thread has read cand; column j holds the pivot column
        const T *vj = A + (long)lda * j;
        const T x0 = vj[j];
        const T alpha = (x0 != T(0)) ? -copysign(nrm, x0) : -nrm;
        const T vhead = x0 - alpha;
        const T vn = vhead * vhead + (nn2 - x0 * x0);
        const int q0 = j - j % VW;   // first 16-byte piece holding row j
        AM<T> mine{-1LL, INT_MAX};
        for (int c = j + 1 + threadIdx.x; c < m; c += ID_NT) {
            T *Ac = A + (long)lda * c;
            T dp[VW] = {};
            for (int q = q0; q < r; q += VW) {
                T a[VW], vv[VW];
                ld16(Ac + q, a);
                ld16(vj + q, vv);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const int i = q + e;
                    if (i >= j && i < r) dp[e] += (i == j ? vhead : vv[e]) * a[e];
                }
            }
            T d = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) d += dp[e];
            const T coef = vn > T(0) ? T(2) * d / vn : T(0);
            T sp[VW] = {};
            for (int q = q0; q < r; q += VW) {
                T a[VW], vv[VW];
                ld16(Ac + q, a);
                ld16(vj + q, vv);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const int i = q + e;
                    if (i >= j && i < r) {
                        a[e] -= coef * (i == j ? vhead : vv[e]);
                        if (i > j) sp[e] += a[e] * a[e];
                    }
                }
                st16(Ac + q, a);
            }
            T sq = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) sq += sp[e];
            const long long kc = nn_key(sq);
            if (kc > mine.v || (kc == mine.v && c < mine.i)) mine = AM<T>{kc, c};
        }
        offer(mine);
        if (threadIdx.x == 0) v[j] = alpha;
        k = j + 1;
    }
    __syncthreads();
    for (int jj = threadIdx.x; jj < k; jj += ID_NT) A[jj + (long)lda * jj] = v[jj];   // R(j, j)
    __syncthreads();
    // T = R11^-1 R12 in place, one thread per column of R12, by columns of R11:
    // t_i = x_i / R_ii, then x_(0..i) -= t_i R(0..i, i)
    auto solve_T_inplace = [&]() {
        for (int c = k + threadIdx.x; c < m; c += ID_NT) {
            T *col = A + (long)lda * c;
            for (int i = k - 1; i >= 0; --i) {
                const T ti = col[i] / A[i + (long)lda * i];
                col[i] = ti;
                const T *Ri = A + (long)lda * i;
                for (int q = 0; q < i; q += VW) {
                    T a[VW], rr[VW];
                    ld16(col + q, a);
                    ld16(Ri + q, rr);
#pragma unroll
                    for (int e = 0; e < VW; ++e)
                        if (q + e < i) a[e] -= ti * rr[e];
                    st16(col + q, a);
                }
            }
        }
        __syncthreads();
    };
    solve_T_inplace();

    // ---- exchanges while some |T_ij| > 2 (largest entry, first in row-major order)
    for (int sw = 0; sw < ID_MAX_SWAPS && k > 0 && k < m; ++sw) {
        const int nc = m - k;
        AM<T> loc{-1LL, INT_MAX};
        for (int q = threadIdx.x; q < k * nc; q += ID_NT) {
            int i = q / nc, jj = q % nc;  // row-major linear index q
            const long long a = abs_key(A[i + (long)lda * (k + jj)]);
            if (a > loc.v || (a == loc.v && q < loc.i)) {
                loc.v = a;
                loc.i = q;
            }
        }
        AM<T> best = blk_argmax(loc, sham);
        if (key_val(best.v, T(0)) <= T(2)) break;
        __syncthreads();
        if (threadIdx.x == 0) {
            int i = best.i / nc, jj = best.i % nc;
            int t = order[i];
            order[i] = order[k + jj];
            order[k + jj] = t;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < m * r; idx += ID_NT) {
            int c = idx / r, i = idx % r;
            A[i + (long)lda * c] = L[order[c] + (long)mcap * i];
        }
        __syncthreads();
        for (int j = 0; j < k; ++j) {
            T part = 0;
            for (int i = j + threadIdx.x; i < r; i += ID_NT) part += A[i + (long)lda * j] * A[i + (long)lda * j];
            T nn = sqrt(blk_sum(part, shs));
            householder_step(A, r, lda, m, j, nn, v, shs);
        }
        solve_T_inplace();
    }

    // ---- outputs
    T *Tm = ws + me.toff;
    for (int idx = threadIdx.x; idx < k * (m - k); idx += ID_NT) {
        int i = idx % k, jj = idx / k;
        Tm[i + (long)kcap * jj] = A[i + (long)lda * (k + jj)];
    }
    if (threadIdx.x == 0) {
        kout[2 * node + side] = k;
        atomicMax(&front_kmax[N.cf], k);
    }
    int *ordg = iws + me.ordoff;
    int *sk = iws + me.skioff;
    const NodeSide sa = leaf ? me : nodes[N.a].s[side];
    const NodeSide sb = leaf ? me : nodes[N.b].s[side];
    for (int c = threadIdx.x; c < m; c += ID_NT) {
        ordg[c] = order[c];
        if (c < k) {
            int o = order[c];
            sk[c] = leaf ? N.lo + o : (o < ka ? iws[sa.skioff + o] : iws[sb.skioff + o - ka]);
        }
    }
    __syncthreads();
    // the local test matrix W (m x r) replaces A in shared memory:
    // rows compress Psi (stream 1), columns Omega (stream 0)
    T *Wl = A;
    const int strm = side == 0 ? 1 : 0;
    for (int idx = threadIdx.x; idx < m * r; idx += ID_NT) {
        int row = idx % m, j = idx / m;
        T val;
        if (leaf)
            val = (T)rademacher(seed, strm, C.box, N.lo + row, j);
        else
            val = row < ka ? ws[sa.tloff + row + (long)sa.kcap * j] : ws[sb.tloff + (row - ka) + (long)sb.kcap * j];
        Wl[row + (long)m * j] = val;
    }
    __syncthreads();
    T *skel = ws + me.skoff;
    T *tl = ws + me.tloff;
    for (int idx = threadIdx.x; idx < k * r; idx += ID_NT) {
        int i = idx % k, j = idx / k;
        skel[i + (long)kcap * j] = L[order[i] + (long)mcap * j];
        const T *wc = Wl + (long)m * j;
        T acc = wc[order[i]];
        for (int jj = 0; jj < m - k; ++jj) acc += Tm[i + (long)kcap * jj] * wc[order[k + jj]];
        tl[i + (long)kcap * j] = acc;
    }
}

// Tall bases, bottom-up: U^tall (|R| x k, ld |R|) of each node side.
template <class T>
__global__ void k_hss_tall(const NodeDev *__restrict__ nodes, const int *__restrict__ work,
                           const int *__restrict__ kout, T *__restrict__ ws, const int *__restrict__ iws) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int node = work[blockIdx.x] >> 1, side = work[blockIdx.x] & 1;
    const NodeDev N = nodes[node];
    const NodeSide me = N.s[side];
    const int k = kout[2 * node + side];
    const int R = N.hi - N.lo;
    const bool leaf = N.a < 0;
    int ka = 0, m = R;
    if (!leaf) {
        ka = kout[2 * N.a + side];
        m = ka + kout[2 * N.b + side];
    }
    int *inv = reinterpret_cast<int *>(smraw);                          // m
    T *Ul = reinterpret_cast<T *>(smraw + sizeof(int) * ((m + 1) & ~1)); // m x k (ld m)
    const int *ord = iws + me.ordoff;
    for (int c = threadIdx.x; c < m; c += blockDim.x) inv[ord[c]] = c;
    __syncthreads();
    const T *Tm = ws + me.toff;
    for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
        int q = idx % m, i = idx / m;
        int p = inv[q];
        Ul[q + (long)m * i] = p < k ? T(p == i ? 1 : 0) : Tm[i + (long)me.kcap * (p - k)];
    }
    __syncthreads();
    T *out = ws + me.talloff;
    if (leaf) {
        for (int idx = threadIdx.x; idx < R * k; idx += blockDim.x) out[idx] = Ul[idx];
        return;
    }
    const NodeSide sa = nodes[N.a].s[side], sb = nodes[N.b].s[side];
    const int Ra = nodes[N.a].hi - nodes[N.a].lo, Rb = nodes[N.b].hi - nodes[N.b].lo;
    const int kb_ = m - ka;
    const T *Ua = ws + sa.talloff, *Ub = ws + sb.talloff;
    for (int idx = threadIdx.x; idx < R * k; idx += blockDim.x) {
        int rho = idx % R, i = idx / R;
        T acc = 0;
        if (rho < Ra) {
            for (int q = 0; q < ka; ++q) acc += Ua[rho + (long)Ra * q] * Ul[q + (long)m * i];
        } else {
            int rr = rho - Ra;
            for (int q = 0; q < kb_; ++q) acc += Ub[rr + (long)Rb * q] * Ul[ka + q + (long)m * i];
        }
        out[idx] = acc;
    }
}

// One 32 x 32 tile of H per CTA, written into the parent front through fmap.
template <class T>
__global__ void k_hss_expand(const ExpandItem *__restrict__ items, const NodeDev *__restrict__ nodes,
                             const int *__restrict__ kout, const ExpandFront *__restrict__ efs,
                             const T *__restrict__ ws, const int *__restrict__ iws, T *__restrict__ arena,
                             T *__restrict__ keep) {
    pdl_launch_next();
    pdl_wait_prev();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T Pm[128 * EXP_TILE];
    const ExpandItem it = items[blockIdx.x];
    const ExpandFront E = efs[it.cf];
    const T *S = reinterpret_cast<const T *>(E.S);
    T *Mp = arena + E.poff;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    if (it.type == 0) {
        for (int yy = ty; yy < EXP_TILE; yy += 8) {
            int i = it.r0 + tx, j = it.c0 + yy;
            if (i >= it.rhi || j >= it.chi) continue;
            T val = S[i + E.lds * j];
            Mp[E.fmap[i] + (long)E.pn * E.fmap[j]] = val;
            if (E.keep_h >= 0) keep[E.keep_h + i + (long)E.nb * j] = val;
        }
        return;
    }
    const NodeDev Na = nodes[it.na], Nb = nodes[it.nb];
    const NodeSide ua = Na.s[0], vb = Nb.s[1];
    const int ka = kout[2 * it.na + 0], kb_ = kout[2 * it.nb + 1];
    const int Ra = Na.hi - Na.lo, Rb = Nb.hi - Nb.lo;
    const T *Ua = ws + ua.talloff, *Vb = ws + vb.talloff;
    const int *Ja = iws + ua.skioff, *Kb = iws + vb.skioff;
    T *Sab = reinterpret_cast<T *>(smraw);          // ka x kb (ld ka)
    T *Vt = Sab + (long)ka * kb_;                   // 32 x kb (ld 32)
    for (int idx = threadIdx.x; idx < ka * kb_; idx += blockDim.x) {
        int q = idx % ka, q2 = idx / ka;
        Sab[idx] = S[Ja[q] + E.lds * Kb[q2]];
    }
    for (int idx = threadIdx.x; idx < EXP_TILE * kb_; idx += blockDim.x) {
        int jj = idx % EXP_TILE, q2 = idx / EXP_TILE;
        int col = it.c0 + jj;
        Vt[idx] = col < it.chi ? Vb[(col - Nb.lo) + (long)Rb * q2] : T(0);
    }
    __syncthreads();
    // Pm = S(J_a, K_b) V^tall_b(cols of this tile)^t   (ka x 32)
    for (int idx = threadIdx.x; idx < ka * EXP_TILE; idx += blockDim.x) {
        int q = idx % ka, jj = idx / ka;
        T acc = 0;
        for (int q2 = 0; q2 < kb_; ++q2) acc += Sab[q + ka * q2] * Vt[jj + EXP_TILE * q2];
        Pm[q + ka * jj] = acc;
    }
    __syncthreads();
    for (int yy = ty; yy < EXP_TILE; yy += 8) {
        int i = it.r0 + tx, j = it.c0 + yy;
        if (i >= it.rhi || j >= it.chi) continue;
        T acc = 0;
        for (int q = 0; q < ka; ++q) acc += Ua[(i - Na.lo) + (long)Ra * q] * Pm[q + ka * yy];
        Mp[E.fmap[i] + (long)E.pn * E.fmap[j]] = acc;
        if (E.keep_h >= 0) keep[E.keep_h + i + (long)E.nb * j] = acc;
    }
}

template <class T>
int launch_hss_id(const NodeDev *nodes, const int *work, int nwork, const CompFront<T> *cf, T *ws, int *iws,
                  int *kout, int *front_kmax, T tol, uint64_t seed, size_t smem, cudaStream_t s) {
    if (nwork == 0) return HSS_OK;
    HSS_SMEM(k_hss_id<T>, 220 * 1024);
    HSS_PROF("hss_id", s);
    HSS_CUDA(launch_pdl(k_hss_id<T>, dim3(nwork), dim3(ID_NT), smem, s, nodes, work, cf, ws, iws, kout, front_kmax, tol, seed));
    HSS_CHECK_LAUNCH("k_hss_id");
    return HSS_OK;
}

template <class T>
int launch_hss_tall(const NodeDev *nodes, const int *work, int nwork, const int *kout, T *ws, int *iws, size_t smem,
                    cudaStream_t s) {
    if (nwork == 0) return HSS_OK;
    HSS_SMEM(k_hss_tall<T>, 220 * 1024);
    HSS_PROF("hss_tall", s);
    HSS_CUDA(launch_pdl(k_hss_tall<T>, dim3(nwork), dim3(256), smem, s, nodes, work, kout, ws, (const int *)iws));
    HSS_CHECK_LAUNCH("k_hss_tall");
    return HSS_OK;
}

template <class T>
int launch_hss_expand(const ExpandItem *items, int nitems, const NodeDev *nodes, const int *kout,
                      const ExpandFront *ef, const T *ws, const int *iws, T *arena, T *keep, int kmax,
                      cudaStream_t s) {
    if (nitems == 0) return HSS_OK;
    HSS_PROF("hss_expand", s);
    HSS_SMEM(k_hss_expand<T>, 160 * 1024);
    // S(J_a,K_b) (kmax x kmax) and a 32 x kmax tile of V^tall
    size_t smem = sizeof(T) * (size_t)(kmax * kmax + EXP_TILE * kmax);
    HSS_CUDA(launch_pdl(k_hss_expand<T>, dim3(nitems), dim3(256), smem, s, items, nodes, kout, ef, ws, iws, arena, keep));
    HSS_CHECK_LAUNCH("k_hss_expand");
    return HSS_OK;
}

// ---------------------------------------------------------------- residual probe
// Per probed front: ||(S - H) W||_F^2 and ||S W||_F^2 for nprobe +-1 columns W
// of stream 2 (the counter generator of the samples).  k_hss_probe: one CTA
// per 128 x 128 tile; thread = row i of S (child front) and of H (parent front,
// rows and columns through fmap), the tile's columns of W generated into shared
// memory; the row's partial sums go to rowacc in FP64.  k_hss_probe_norms: one
// CTA per front sums the squares of the finished row sums.
template <class T>
__global__ void __launch_bounds__(PROBE_NT) k_hss_probe(const ProbeItem *__restrict__ items,
                                                        const ExpandFront *__restrict__ ef,
                                                        const T *__restrict__ arena, uint64_t seed, int nprobe,
                                                        double *__restrict__ rowacc) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ T w[PROBE_NT * PROBE_MAX];
    __shared__ long hcol[PROBE_NT];
    const ProbeItem it = items[blockIdx.x];
    const ExpandFront E = ef[it.f];
    const T *S = static_cast<const T *>(E.S);
    const T *Mp = arena + E.poff;
    const int jn = min(PROBE_NT, E.nb - it.col0);
    for (int e = threadIdx.x; e < jn * nprobe; e += PROBE_NT) {
        const int jj = e / nprobe, q = e - jj * nprobe;
        w[jj * PROBE_MAX + q] = (T)rademacher(seed, 2, it.box, it.col0 + jj, q);
    }
    for (int jj = threadIdx.x; jj < jn; jj += PROBE_NT) hcol[jj] = (long)E.pn * E.fmap[it.col0 + jj];
    __syncthreads();
    const int i = it.row0 + (int)threadIdx.x;
    if (i >= E.nb) return;
    const T *Hr = Mp + E.fmap[i];
    const T *Sr = S + i + E.lds * (long)it.col0;
    T sw[PROBE_MAX], dw[PROBE_MAX];
#pragma unroll
    for (int q = 0; q < PROBE_MAX; ++q) sw[q] = dw[q] = T(0);
#pragma unroll 8
    for (int jj = 0; jj < jn; ++jj) {
        const T sv = Sr[E.lds * jj];
        const T dv = sv - Hr[hcol[jj]];
#pragma unroll
        for (int q = 0; q < PROBE_MAX; ++q)
            if (q < nprobe) {
                const T wq = w[jj * PROBE_MAX + q];
                sw[q] = fma(sv, wq, sw[q]);
                dw[q] = fma(dv, wq, dw[q]);
            }
    }
    // this column tile's share of row i: region [column tile][row][2 x PROBE_MAX]
    double *ra = rowacc + it.rowacc + ((long)(it.col0 / PROBE_NT) * E.nb + i) * 2 * PROBE_MAX;
#pragma unroll
    for (int q = 0; q < PROBE_MAX; ++q)
        if (q < nprobe) {
            ra[q] = (double)sw[q];
            ra[PROBE_MAX + q] = (double)dw[q];
        }
}

__global__ void __launch_bounds__(PROBE_NT) k_hss_probe_norms(const ProbeFront *__restrict__ pf,
                                                              const ExpandFront *__restrict__ ef, int nprobe,
                                                              const double *__restrict__ rowacc,
                                                              double *__restrict__ acc) {
    pdl_launch_next();
    pdl_wait_prev();
    __shared__ double red[2][PROBE_NT / 32];
    const ProbeFront P = pf[blockIdx.x];
    const int nb = ef[P.f].nb, ntc = (nb + PROBE_NT - 1) / PROBE_NT;
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < nb; i += PROBE_NT)
        for (int q = 0; q < nprobe; ++q) {
            double sv = 0.0, dv = 0.0;
            for (int ct = 0; ct < ntc; ++ct) {   // column tiles in order: a fixed summation order
                const double *ra = rowacc + P.rowacc + ((long)ct * nb + i) * 2 * PROBE_MAX;
                sv += ra[q];
                dv += ra[PROBE_MAX + q];
            }
            den += sv * sv;
            num += dv * dv;
        }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = num;
        red[1][wid] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < PROBE_NT / 32; ++k) {
            a += red[0][k];
            b += red[1][k];
        }
        acc[2 * blockIdx.x] = a;
        acc[2 * blockIdx.x + 1] = b;
    }
}

template <class T>
int launch_hss_probe(const ProbeItem *items, int nitems, const ProbeFront *pf, int nfronts, const ExpandFront *ef,
                     const T *arena, uint64_t seed, int nprobe, double *rowacc, double *acc, cudaStream_t s) {
    if (nitems == 0) return HSS_OK;
    {
        HSS_PROF("hss_probe", s);
        HSS_CUDA(launch_pdl(k_hss_probe<T>, dim3(nitems), dim3(PROBE_NT), 0, s, items, ef, arena, seed, nprobe, rowacc));
    }
    {
        HSS_PROF("hss_probe", s);
        HSS_CUDA(launch_pdl(k_hss_probe_norms, dim3(nfronts), dim3(PROBE_NT), 0, s, pf, ef, nprobe, rowacc, acc));
    }
    HSS_CHECK_LAUNCH("k_hss_probe");
    return HSS_OK;
}

#define INST(T)                                                                                                \
    template int launch_hss_probe<T>(const ProbeItem *, int, const ProbeFront *, int, const ExpandFront *,      \
                                     const T *, uint64_t, int, double *, double *, cudaStream_t);               \
    template int launch_hss_id<T>(const NodeDev *, const int *, int, const CompFront<T> *, T *, int *, int *,  \
                                  int *, T, uint64_t, size_t, cudaStream_t);                                  \
    template int launch_hss_tall<T>(const NodeDev *, const int *, int, const int *, T *, int *, size_t,        \
                                    cudaStream_t);                                                             \
    template int launch_hss_expand<T>(const ExpandItem *, int, const NodeDev *, const int *, const ExpandFront *, \
                                      const T *, const int *, T *, T *, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace hssnd
