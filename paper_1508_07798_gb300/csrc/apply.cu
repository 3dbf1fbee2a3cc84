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

#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>

namespace hssnd {

constexpr int AP_NT = 256;
constexpr int AP_WPB = AP_NT / 32;   // warps (work items) per CTA


// One warp per work item = (front, 32-row tile, column chunk of at most
// APPLY_CHUNK columns).  Lane l owns row row0 + l; x is gathered one value per
// lane and broadcast by shuffles; 32 matrix loads per lane are in flight per
// group of 32 columns.  A tile split over several chunks writes partial sums;
// the last warp to finish (atomic ticket) adds them in chunk order and writes
// the result, so the sum order is fixed.  No barrier, no waiting.
//   FWD: y = [F_ii^-1 P^t ; -F_bi F_ii^-1 P^t] x(Iperm)  ->  t = y[0,ni), x_B += y[ni,n)
//   BWD: x_I = t - W x_B
// The products of one work item: lane l's sums for row row0 + l.
template <class T, int RB, bool FWD>
__device__ __forceinline__ void apply_item_sums(const ApplyItem &it, const FrontDev &F, const T *__restrict__ arena,
                                                const int *__restrict__ iperm, const int *__restrict__ blist,
                                                const double *__restrict__ w, long ldw, int nrhs, T (&acc)[RB]) {
    const int lane = threadIdx.x & 31;
    const T *M = arena + F.foff;
    const int colbase = FWD ? 0 : F.ni, nrows = FWD ? F.n : F.ni;
    const int i = it.row0 + lane;
    const bool rowok = i < nrows;
    // arithmetic in the factor's precision (FP32 factors: FP32 products and sums;
    // GB300's FP64 pipe is a small fraction of its FP32 rate)
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = T(0);
    bool waited = false;
    for (int cg = it.c0; cg < it.c1; cg += 32) {
        const int c = cg + lane;
        T m[32];
        const T *col = M + i + (long)F.n * (colbase + cg);
#pragma unroll
        for (int q = 0; q < 32; ++q) m[q] = (rowok && cg + q < it.c1) ? col[(long)F.n * q] : T(0);
        const int dof = c < it.c1 ? (FWD ? iperm[F.iperm_off + c] : blist[F.bset_off + c]) : -1;
        if (!waited) {   // the vectors are the previous kernel's output
            pdl_wait_prev();
            waited = true;
        }
        T z[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) z[r] = (dof >= 0 && r < nrhs) ? (T)w[dof + ldw * r] : T(0);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[r] = fma(m[q], __shfl_sync(0xffffffffu, z[r], q), acc[r]);
        }
    }
}

// The results of one work item (row row0 + lane):
//   FWD: rows [0, ni) to t, rows [ni, n) added into x_B;  BWD: x_I = t - sums
template <class T, int RB, bool FWD>
__device__ __forceinline__ void apply_item_store(const ApplyItem &it, const FrontDev &F, const int *__restrict__ ilist,
                                                 const int *__restrict__ blist, double *__restrict__ w, long ldw,
                                                 double *__restrict__ tv, long ldt, int nrhs, const T (&acc)[RB]) {
    const int i = it.row0 + (threadIdx.x & 31);
    if (i >= (FWD ? F.n : F.ni)) return;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (r >= nrhs) break;
        const double y = (double)acc[r];
        if (FWD) {
            if (i < F.ni)
                tv[ilist[F.iset_off + i] + ldt * r] = y;
            else
                w[blist[F.bset_off + i - F.ni] + ldw * r] += y;
        } else {
            const int dof = ilist[F.iset_off + i];
            w[dof + ldw * r] = tv[dof + ldt * r] - y;
        }
    }
}

// One warp per work item = (front, 32-row tile, column chunk of at most
// APPLY_CHUNK columns).  Lane l owns row row0 + l; x is gathered one value per
// lane and broadcast by shuffles; 32 matrix loads per lane are in flight per
// group of 32 columns.  A tile split over several chunks writes partial sums;
// the last warp to finish (atomic ticket) adds them in chunk order and writes
// the result, so the sum order is fixed.  No barrier, no waiting.
//   FWD: y = [F_ii^-1 P^t ; -F_bi F_ii^-1 P^t] x(Iperm)  ->  t = y[0,ni), x_B += y[ni,n)
//   BWD: x_I = t - W x_B
template <class T, int RB, bool FWD>
__global__ void __launch_bounds__(AP_NT) k_apply(const ApplyItem *__restrict__ items, int nitems,
                                               const FrontDev *__restrict__ fr, const T *__restrict__ arena,
                                               const int *__restrict__ iperm, const int *__restrict__ ilist,
                                               const int *__restrict__ blist, const ApplyParams *__restrict__ prm,
                                               double *__restrict__ part, int *__restrict__ tickets) {
    pdl_launch_next();
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * AP_WPB + (threadIdx.x >> 5);
    if (item >= nitems) return;   // whole warps leave together
    const ApplyItem it = items[item];
    const FrontDev F = fr[it.front];
    T acc[RB];
    apply_item_sums<T, RB, FWD>(it, F, arena, iperm, blist, prm->w, prm->ldw, prm->nrhs, acc);
    pdl_wait_prev();   // (an item without columns has not waited yet)
    if (it.nchunk > 1) {
        T *mine = reinterpret_cast<T *>(part) + (long)item * 32 * RB;
#pragma unroll
        for (int r = 0; r < RB; ++r) mine[r * 32 + lane] = acc[r];
        __threadfence();
        int ticket = 0;
        if (lane == 0) ticket = atomicAdd(&tickets[it.tile], 1);
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        if (ticket != it.nchunk - 1) return;
        __threadfence();
        const T *first = reinterpret_cast<const T *>(part) + (long)it.first * 32 * RB;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            T y = T(0);
            for (int ch = 0; ch < it.nchunk; ++ch) y += __ldcg(first + (long)ch * 32 * RB + r * 32 + lane);
            acc[r] = y;
        }
        if (lane == 0) tickets[it.tile] = 0;   // ready for the next apply
    }
    apply_item_store<T, RB, FWD>(it, F, ilist, blist, prm->w, prm->ldw, prm->tv, prm->ldt, prm->nrhs, acc);
}

// The deepest levels as one launch: CTA s walks the stages of subtree s (the
// fronts below its root in stage nst - 1), deepest stage first forward and
// root first backward, its eight warps taking the stage's items (one 32-row
// tile, every column) and a block barrier between stages.  Subtrees hold
// disjoint dofs (DG dofs belong to elements), so the CTAs never meet; inside
// one, the barrier orders a stage's writes of x before the next stage's reads.
template <class T, int RB, bool FWD>
__global__ void __launch_bounds__(AP_NT) k_apply_sub(const ApplyItem *__restrict__ items, const int *__restrict__ off,
                                                   int nst, const FrontDev *__restrict__ fr, const T *__restrict__ arena,
                                                   const int *__restrict__ iperm, const int *__restrict__ ilist,
                                                   const int *__restrict__ blist, const ApplyParams *__restrict__ prm) {
    pdl_launch_next();
    const int sub = blockIdx.x, warp = threadIdx.x >> 5;
    double *w = prm->w;
    double *tv = prm->tv;
    const long ldw = prm->ldw, ldt = prm->ldt;
    const int nrhs = prm->nrhs;
    for (int l = 0; l < nst; ++l) {
        const int q = FWD ? l : nst - 1 - l;
        const int b = off[sub * (nst + 1) + q], e = off[sub * (nst + 1) + q + 1];
        for (int k = b + warp; k < e; k += AP_WPB) {
            const ApplyItem it = items[k];
            const FrontDev F = fr[it.front];
            T acc[RB];
            apply_item_sums<T, RB, FWD>(it, F, arena, iperm, blist, w, ldw, nrhs, acc);
            pdl_wait_prev();
            apply_item_store<T, RB, FWD>(it, F, ilist, blist, w, ldw, tv, ldt, nrhs, acc);
        }
        pdl_wait_prev();   // warps without items
        __syncthreads();
    }
}

__global__ void k_apply_set(ApplyParams *d, ApplyParams v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d = v;
}

// w = x (every right-hand side), skipped when they alias
__global__ void k_apply_copyin(const ApplyParams *__restrict__ prm, long N) {
    pdl_launch_next();
    const double *x = prm->x;
    double *w = prm->w;
    if (x == w) return;
    long tot = N * prm->nrhs;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < tot; g += (long)gridDim.x * blockDim.x) {
        long r = g / N, i = g % N;
        w[i + prm->ldw * r] = x[i + prm->ldx * r];
    }
}

// The whole sweep (copy-in, forward levels, top block, backward levels) as
// one kernel sequence on stream s, each launch overlapping the previous one's
// tail (launch_pdl); parameters come from f->d_aparams.
template <class T, int RB> static int record_sweep(const hss_factor_t *f, cudaStream_t s, int &nk) {
    const T *arena = f->arena_ptr<T>();
    const ApplyParams *prm = f->d_aparams.as<ApplyParams>();
    nk = 0;
    k_apply_copyin<<<2 * device_sms(), 256, 0, s>>>(prm, f->ndof);
    ++nk;
    cudaError_t e = cudaSuccess;
    auto sub = [&](bool fwd) {
        if (f->sub_nst == 0 || e != cudaSuccess) return;
        const int *il = f->tree->d_iset.as<int>(), *bl = f->tree->d_bset.as<int>();
        if (fwd)
            e = launch_pdl(k_apply_sub<T, RB, true>, dim3(f->sub_n), dim3(AP_NT), 0, s, (const ApplyItem *)f->d_sub_fwd,
                           (const int *)f->d_sub_off_fwd, f->sub_nst, (const FrontDev *)f->d_sub_fronts, arena,
                           (const int *)f->d_iperm.as<int>(), il, bl, prm);
        else
            e = launch_pdl(k_apply_sub<T, RB, false>, dim3(f->sub_n), dim3(AP_NT), 0, s, (const ApplyItem *)f->d_sub_bwd,
                           (const int *)f->d_sub_off_bwd, f->sub_nst, (const FrontDev *)f->d_sub_fronts, arena,
                           (const int *)f->d_iperm.as<int>(), il, bl, prm);
        ++nk;
    };
    for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        if (fwd) sub(true);
        for (size_t k = 0; k < f->apply.size(); ++k) {
            const size_t q = fwd ? k : f->apply.size() - 1 - k;
            if ((int)q < f->sub_nst) continue;   // in the subtree launch
            const ApplyStage &st = f->apply[q];
            const int *ilist = st.top ? f->d_topset.as<int>() : f->tree->d_iset.as<int>();
            const int nt = fwd ? st.nfwd : st.nbwd;
            if (nt == 0) continue;
            const ApplyItem *itm = fwd ? st.d_fwd : st.d_bwd;
            double *part = f->d_apart.as<double>() + (fwd ? st.part_fwd : st.part_bwd) * 32 * APPLY_RB;
            int *tk = f->d_tickets.as<int>() + (fwd ? st.tk_fwd : st.tk_bwd);
            if (e != cudaSuccess) break;
            if (fwd)
                e = launch_pdl(k_apply<T, RB, true>, dim3(cdiv(nt, AP_WPB)), dim3(AP_NT), 0, s, itm, nt, (const FrontDev *)st.d_fronts,
                               arena, (const int *)f->d_iperm.as<int>(), ilist, (const int *)f->tree->d_bset.as<int>(),
                               prm, part, tk);
            else
                e = launch_pdl(k_apply<T, RB, false>, dim3(cdiv(nt, AP_WPB)), dim3(AP_NT), 0, s, itm, nt, (const FrontDev *)st.d_fronts,
                               arena, (const int *)f->d_iperm.as<int>(), ilist, (const int *)f->tree->d_bset.as<int>(),
                               prm, part, tk);
            ++nk;
        }
        if (!fwd) sub(false);
    }
    if (e != cudaSuccess) return cuda_fail(e, "apply sweep launch");
    HSS_CHECK_LAUNCH("apply sweep");
    return HSS_OK;
}

// Work items of one sweep direction of a stage: 32-row tiles, each split into
// column chunks of `chunk` (pass 0: forward, n rows x ni columns; pass 1:
// backward, ni rows x nb columns).
static void stage_items(const ApplyStage &st, int pass, int chunk, std::vector<ApplyItem> &items, int &tiles) {
    items.clear();
    tiles = 0;
    for (int f = 0; f < (int)st.h_fronts.size(); ++f) {
        const FrontDev &d = st.h_fronts[f];
        if (d.ni == 0) continue;
        const int nrows = pass == 0 ? d.n : d.ni;
        const int ncols = pass == 0 ? d.ni : d.nb;
        const int nch = std::max(1, cdiv(ncols, chunk));
        for (int r0 = 0; r0 < nrows; r0 += 32) {
            const int first = (int)items.size();
            const int tile = nch > 1 ? tiles++ : -1;
            for (int ch = 0; ch < nch; ++ch)
                items.push_back({f, r0, std::min(ncols, ch * chunk), std::min(ncols, (ch + 1) * chunk), tile, first, nch});
        }
    }
}

int pack_apply(hss_factor_t *F, cudaStream_t s) {
    for (auto &g : F->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    const size_t nst = F->apply.size();
    std::vector<std::vector<ApplyItem>> items(2 * nst);
    long part_total = 0;
    int tk_total = 0;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t bytes = 0;
    for (size_t q = 0; q < nst; ++q) {
        ApplyStage &st = F->apply[q];
        int tiles[2];
        for (int pass = 0; pass < 2; ++pass) stage_items(st, pass, st.chunk[pass], items[2 * q + pass], tiles[pass]);
        st.nfwd = (int)items[2 * q].size();
        st.nbwd = (int)items[2 * q + 1].size();
        st.part_fwd = part_total;
        part_total += st.nfwd;
        st.part_bwd = part_total;
        part_total += st.nbwd;
        st.tk_fwd = tk_total;
        tk_total += tiles[0];
        st.tk_bwd = tk_total;
        tk_total += tiles[1];
        bytes += al(sizeof(FrontDev) * st.h_fronts.size()) + al(sizeof(ApplyItem) * st.nfwd) +
                 al(sizeof(ApplyItem) * st.nbwd);
    }
    // subtree part: root stage = the shallowest stage (below the top block)
    // with at least APPLY_SUB_MIN fronts, none larger than APPLY_SUB_MAXN
    // (this and every deeper stage); every front of the stages up to it
    // belongs to the subtree of its ancestor in the root stage
    int qr = -1;
    for (size_t q = 0; q < nst; ++q) {
        if (F->apply[q].top) break;
        int nmax = 0;
        for (const FrontDev &d : F->apply[q].h_fronts) nmax = std::max(nmax, d.n);
        if (nmax > APPLY_SUB_MAXN) break;   // larger fronts need the level launch's parallelism
        if (F->apply[q].nfronts >= APPLY_SUB_MIN) qr = (int)q;
    }
    std::vector<FrontDev> sfr;
    std::vector<ApplyItem> sit[2];
    std::vector<int> soff[2];
    F->sub_nst = 0;
    F->sub_n = 0;
    if (qr >= 1) {
        const hss_tree *t = F->tree;
        const int nsub = (int)F->apply[qr].h_fronts.size();
        const int root_level = t->level[F->apply[qr].h_fronts[0].box];
        std::unordered_map<int, int> sub_of_root;
        for (int f = 0; f < nsub; ++f) sub_of_root[F->apply[qr].h_fronts[f].box] = f;
        // per subtree and stage, its fronts
        std::vector<std::vector<int>> lists((size_t)nsub * (qr + 1));
        for (int q = 0; q <= qr; ++q) {
            const ApplyStage &st = F->apply[q];
            for (int f = 0; f < (int)st.h_fronts.size(); ++f) {
                int b = st.h_fronts[f].box;
                while (b >= 0 && t->level[b] > root_level) b = t->parent[b];
                const auto it = sub_of_root.find(b);
                if (it == sub_of_root.end()) {   // not below a root (cannot happen in a box tree)
                    qr = -1;
                    break;
                }
                lists[(size_t)it->second * (qr + 1) + q].push_back((int)sfr.size());
                sfr.push_back(st.h_fronts[f]);
            }
            if (qr < 0) break;
        }
        if (qr >= 1) {
            for (int pass = 0; pass < 2; ++pass) {
                soff[pass].assign((size_t)nsub * (qr + 2), 0);
                for (int sb = 0; sb < nsub; ++sb)
                    for (int q = 0; q <= qr; ++q) {
                        soff[pass][(size_t)sb * (qr + 2) + q] = (int)sit[pass].size();
                        for (int fi : lists[(size_t)sb * (qr + 1) + q]) {
                            const FrontDev &d = sfr[fi];
                            if (d.ni == 0) continue;
                            const int nrows = pass == 0 ? d.n : d.ni, ncols = pass == 0 ? d.ni : d.nb;
                            for (int r0 = 0; r0 < nrows; r0 += 32)
                                sit[pass].push_back({fi, r0, 0, ncols, -1, (int)sit[pass].size(), 1});
                        }
                        soff[pass][(size_t)sb * (qr + 2) + q + 1] = (int)sit[pass].size();
                    }
            }
            F->sub_nst = qr + 1;
            F->sub_n = nsub;
            bytes += al(sizeof(FrontDev) * sfr.size()) + al(sizeof(ApplyItem) * sit[0].size()) +
                     al(sizeof(ApplyItem) * sit[1].size()) + al(sizeof(int) * soff[0].size()) +
                     al(sizeof(int) * soff[1].size());
        }
    }
    // every stage's fronts and work items in one device allocation
    std::vector<char> pack(std::max(bytes, (size_t)1));
    int rc;
    if ((rc = F->apply_buf.alloc(pack.size()))) return rc;
    size_t o = 0;
    char *base = F->apply_buf.as<char>();
    auto put = [&](const void *src, size_t b) -> char * {
        if (b) std::memcpy(pack.data() + o, src, b);
        char *d = base + o;
        o += al(b);
        return d;
    };
    for (size_t q = 0; q < nst; ++q) {
        ApplyStage &st = F->apply[q];
        st.d_fronts = reinterpret_cast<FrontDev *>(put(st.h_fronts.data(), sizeof(FrontDev) * st.h_fronts.size()));
        st.d_fwd = reinterpret_cast<ApplyItem *>(put(items[2 * q].data(), sizeof(ApplyItem) * st.nfwd));
        st.d_bwd = reinterpret_cast<ApplyItem *>(put(items[2 * q + 1].data(), sizeof(ApplyItem) * st.nbwd));
    }
    if (F->sub_nst > 0) {
        F->d_sub_fronts = reinterpret_cast<FrontDev *>(put(sfr.data(), sizeof(FrontDev) * sfr.size()));
        F->d_sub_fwd = reinterpret_cast<ApplyItem *>(put(sit[0].data(), sizeof(ApplyItem) * sit[0].size()));
        F->d_sub_bwd = reinterpret_cast<ApplyItem *>(put(sit[1].data(), sizeof(ApplyItem) * sit[1].size()));
        F->d_sub_off_fwd = reinterpret_cast<int *>(put(soff[0].data(), sizeof(int) * soff[0].size()));
        F->d_sub_off_bwd = reinterpret_cast<int *>(put(soff[1].data(), sizeof(int) * soff[1].size()));
    }
    HSS_CUDA(cudaMemcpyAsync(base, pack.data(), pack.size(), cudaMemcpyHostToDevice, s));
    if ((rc = F->d_apart.alloc(sizeof(double) * 32 * APPLY_RB * std::max(part_total, 1L))) ||
        (rc = F->d_tickets.alloc(sizeof(int) * std::max(tk_total, 1))))
        return rc;
    HSS_CUDA(cudaMemsetAsync(F->d_tickets.p, 0, sizeof(int) * std::max(tk_total, 1), s));
    // (a copy from pageable memory has left `pack` by the time cudaMemcpyAsync returns)
    return HSS_OK;
}

// One sweep with events around every stage launch (the same launches as the
// captured graph for one right-hand side); ms[2 * q + pass] = that launch's time.
template <class T> static int timed_sweep(const hss_factor_t *f, cudaStream_t s, std::vector<cudaEvent_t> &ev,
                                          std::vector<float> &ms) {
    const T *arena = f->arena_ptr<T>();
    const ApplyParams *prm = f->d_aparams.as<ApplyParams>();
    const size_t nst = f->apply.size();
    k_apply_copyin<<<2 * device_sms(), 256, 0, s>>>(prm, f->ndof);
    for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        for (size_t k = 0; k < nst; ++k) {
            const size_t q = fwd ? k : nst - 1 - k;
            const ApplyStage &st = f->apply[q];
            const int nt = fwd ? st.nfwd : st.nbwd;
            if (nt == 0) continue;
            const int *ilist = st.top ? f->d_topset.as<int>() : f->tree->d_iset.as<int>();
            double *part = f->d_apart.as<double>() + (fwd ? st.part_fwd : st.part_bwd) * 32 * APPLY_RB;
            int *tk = f->d_tickets.as<int>() + (fwd ? st.tk_fwd : st.tk_bwd);
            HSS_CUDA(cudaEventRecord(ev[2 * (2 * q + pass)], s));
            if (fwd)
                k_apply<T, 1, true><<<cdiv(nt, AP_WPB), AP_NT, 0, s>>>(st.d_fwd, nt, st.d_fronts, arena,
                                                                       f->d_iperm.as<int>(), ilist,
                                                                       f->tree->d_bset.as<int>(), prm, part, tk);
            else
                k_apply<T, 1, false><<<cdiv(nt, AP_WPB), AP_NT, 0, s>>>(st.d_bwd, nt, st.d_fronts, arena,
                                                                        f->d_iperm.as<int>(), ilist,
                                                                        f->tree->d_bset.as<int>(), prm, part, tk);
            HSS_CUDA(cudaEventRecord(ev[2 * (2 * q + pass) + 1], s));
        }
    }
    HSS_CHECK_LAUNCH("timed apply sweep");
    HSS_CUDA(cudaStreamSynchronize(s));
    for (size_t q = 0; q < nst; ++q)
        for (int pass = 0; pass < 2; ++pass) {
            const ApplyStage &st = f->apply[q];
            if ((pass == 0 ? st.nfwd : st.nbwd) == 0) continue;
            float t = 0;
            HSS_CUDA(cudaEventElapsedTime(&t, ev[2 * (2 * q + pass)], ev[2 * (2 * q + pass) + 1]));
            ms[2 * q + pass] = t;
        }
    return HSS_OK;
}

// Process-wide choices of the tuner: (precision, direction, stage shape) -> chunk.
static std::mutex g_tune_mu;
static std::unordered_map<uint64_t, int> g_tune;

static uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t stage_key(const ApplyStage &st, int pass, int precision) {
    uint64_t h = mix64(0x9e3779b97f4a7c15ULL + (uint64_t)(precision * 4 + pass * 2 + (st.top ? 1 : 0)));
    for (const FrontDev &d : st.h_fronts)
        h = mix64(h ^ (((uint64_t)d.n << 42) | ((uint64_t)d.ni << 21) | (uint64_t)d.nb));
    return h;
}

int tune_apply(hss_factor_t *F, cudaStream_t s) {
    static const int cand[] = {32, 64, 128, 256};
    const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    const size_t nst = F->apply.size();
    std::vector<uint64_t> key(2 * nst);
    bool all_known = true;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (size_t q = 0; q < nst; ++q)
            for (int pass = 0; pass < 2; ++pass) {
                key[2 * q + pass] = stage_key(F->apply[q], pass, F->precision);
                auto it = g_tune.find(key[2 * q + pass]);
                if (it != g_tune.end()) F->apply[q].chunk[pass] = it->second;
                else all_known = false;
            }
    }
    if (all_known) return pack_apply(F, s);
    int rc;
    DevBuf yb;
    if ((rc = F->tvec.alloc(sizeof(double) * (size_t)F->ndof * APPLY_RB)) ||
        (rc = F->d_aparams.alloc(sizeof(ApplyParams))) || (rc = yb.alloc(sizeof(double) * (size_t)F->ndof)))
        return rc;
    HSS_CUDA(cudaMemsetAsync(yb.p, 0, sizeof(double) * F->ndof, s));
    HSS_CUDA(cudaMemsetAsync(F->tvec.p, 0, sizeof(double) * F->ndof, s));
    ApplyParams pv{yb.as<double>(), (long)F->ndof, yb.as<double>(), (long)F->ndof, F->tvec.as<double>(),
                   (long)F->ndof, 1};
    k_apply_set<<<1, 32, 0, s>>>(F->d_aparams.as<ApplyParams>(), pv);
    HSS_CHECK_LAUNCH("k_apply_set");
    std::vector<cudaEvent_t> ev(4 * nst, nullptr);
    for (auto &e : ev) HSS_CUDA(cudaEventCreate(&e));
    std::vector<float> best(2 * nst, 1e30f), ms(2 * nst, 0.f);
    std::vector<int> pick(2 * nst, APPLY_CHUNK);
    for (int c = 0; c < ncand && rc == HSS_OK; ++c) {
        for (auto &st : F->apply) st.chunk[0] = st.chunk[1] = cand[c];
        if ((rc = pack_apply(F, s))) break;
        std::vector<float> mn(2 * nst, 1e30f);
        for (int rep = 0; rep < 3 && rc == HSS_OK; ++rep) {   // the first sweep warms up; keep the fastest
            rc = F->precision == HSS_FP32 ? timed_sweep<float>(F, s, ev, ms) : timed_sweep<double>(F, s, ev, ms);
            if (rep > 0)
                for (size_t i = 0; i < mn.size(); ++i) mn[i] = std::min(mn[i], ms[i]);
        }
        for (size_t i = 0; i < mn.size(); ++i)
            if (mn[i] < best[i]) {
                best[i] = mn[i];
                pick[i] = cand[c];
            }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (size_t q = 0; q < nst; ++q)
            for (int pass = 0; pass < 2; ++pass) {
                F->apply[q].chunk[pass] = pick[2 * q + pass];
                g_tune[key[2 * q + pass]] = pick[2 * q + pass];
            }
    }
    return pack_apply(F, s);
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
        rc = slot == 0 ? record_sweep<T, 1>(f, cs, nk) : record_sweep<T, APPLY_RB>(f, cs, nk);
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
    if ((rc = mf->tvec.alloc(sizeof(double) * (size_t)f->ndof * std::min(nrhs, APPLY_RB)))) return rc;
    if ((rc = mf->d_aparams.alloc(sizeof(ApplyParams)))) return rc;
    const int slot = nrhs == 1 ? 0 : 1;
    if (!f->gexec[slot]) {
        rc = f->precision == HSS_FP32 ? build_graph<float>(mf, slot) : build_graph<double>(mf, slot);
        if (rc) return rc;
    }
    HSS_PROF("apply", s, f->apply_bytes(nrhs));
    for (int k = 0; k < nrhs; k += APPLY_RB) {   // one sweep per block of up to APPLY_RB right-hand sides
        ApplyParams pv{x + ldx * k, ldx, y + ldy * k, ldy, mf->tvec.as<double>(), (long)f->ndof,
                       std::min(APPLY_RB, nrhs - k)};
        prof_add_launches(f->graph_kernels[slot]);
        k_apply_set<<<1, 32, 0, s>>>(mf->d_aparams.as<ApplyParams>(), pv);
        HSS_CHECK_LAUNCH("k_apply_set");
        HSS_CUDA(cudaGraphLaunch(f->gexec[slot], s));
    }
    return HSS_OK;
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_factor_apply_plan(const hss_factor_t *f, int cap, int *chunk_fwd, int *chunk_bwd) {
    if (!f || cap < 0) {
        set_error("hss_factor_apply_plan: invalid argument");
        return -HSS_EINVAL;
    }
    const int n = (int)f->apply.size();
    for (int q = 0; q < std::min(n, cap); ++q) {
        if (chunk_fwd) chunk_fwd[q] = f->apply[q].chunk[0];
        if (chunk_bwd) chunk_bwd[q] = f->apply[q].chunk[1];
    }
    return n;
}

extern "C" int hss_apply(const hss_factor_t *f, int nrhs, const double *x, int ldx, double *y, int ldy,
                         void *stream) {
    if (!f || !x || !y || nrhs < 0 || ldx < f->ndof || ldy < f->ndof) {
        set_error("hss_apply: invalid argument");
        return HSS_EINVAL;
    }
    if (nrhs == 0) return HSS_OK;
    return apply_factor(f, nrhs, x, ldx, y, ldy, (cudaStream_t)stream);
}
