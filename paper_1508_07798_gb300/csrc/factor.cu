// hss_factor: Algorithm 2 of the paper, level by level on the device.
//
//   for each level, deepest first:
//     assemble the fronts [I ; B]            (leaf: A; parent: A(B^mu,B^nu), H^mu/H^nu already in)
//     Gauss-Jordan sweep over the I pivots   -> F_ii^-1, -F_bi F_ii^-1, W, S   (eq. (32))
//     randomized HSS of every S              (Theorem 1; rank-adaptive sample width)
//     expand H into the parent front         (eq. (32)) / the top block (eq. (36))
//   invert the top block A^(0)
//
// The host only schedules: it builds per-level work lists from the tree and
// reads back one small array per sampling round (node ranks and pivot
// status) to decide sample growth and to size the expansion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <cstdint>
#include <cstring>

#include "factor.h"
#include "hss.h"
#include "prof.h"

namespace hssnd {

// A blocking read-back of the factorization (ranks of a sampling round, probe
// norms, pivot flags): the copy and the stream synchronize, counted, with the
// host time spent in them (a copy to pageable memory already waits for the
// stream), so that the host's share of a factorization can be told from the
// device's.
static int factor_readback(void *dst, const void *src, size_t bytes, cudaStream_t s, hss_factor_t *F) {
    HSS_HOST("readback");
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (F) {
        F->host_syncs++;
        F->host_sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    prof_mark_readback();
    return e == cudaSuccess ? HSS_OK : cuda_fail(e, "device read-back");
}

namespace {

// flag = 1 when some stored value of A is NaN or infinite (the block count
// comes from row_ptr[nb] on the device, so the host needs no read-back)
__global__ void k_check_finite(const int *__restrict__ row_ptr, int nb, int bs2, const double *__restrict__ val,
                               int *__restrict__ flag) {
    pdl_launch_next();
    pdl_wait_prev();
    const long tot = (long)row_ptr[nb] * bs2;
    bool bad = false;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < tot; g += (long)gridDim.x * blockDim.x)
        bad |= !isfinite(val[g]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

template <class T> struct StageCtx {
    std::vector<FrontDev> fronts;       // stage-local fronts
    std::vector<int> boxes;             // box of each front (-1: top)
    std::vector<long> parent_off;       // arena offset of the parent front
    std::vector<int> parent_n;
    DevBuf d_status;
};

template <class T>
int assemble_stage(const hss_bsr *A, const hss_tree *t, const std::vector<FrontDev> &fr, const FrontDev *d_fr,
                   const std::vector<std::vector<int>> &dofs, const std::vector<std::vector<int>> &sides,
                   int *elem_slot, T *arena, Work &W, cudaStream_t s) {
    std::vector<StageElem> se;
    int bs = t->bs;
    for (size_t f = 0; f < fr.size(); ++f) {
        const auto &d = dofs[f];
        for (size_t pos = 0; pos < d.size(); pos += bs) se.push_back({d[pos] / bs, (int)f, (int)pos, sides[f][pos / bs]});
    }
    if (se.empty()) return HSS_OK;
    StageElem *d_se;
    int rc;
    if ((rc = W.up(se, &d_se))) return rc;
    return launch_scatter_A<T>(A, d_se, (int)se.size(), elem_slot, d_fr, arena, s);
}

// GEMM engine of a factorization: SIMT FMA, or (FP32 form) tcgen05 TF32
// tensor cores.
struct Engine {
    int tc = 0;          // tensor_cores option: 0 SIMT; 1 TF32 hi/lo split; 2 single TF32; 3 chosen by timing
    int bf16 = 0;        // sample_bf16 option: sampling products on tcgen05 kind::f16, A in three BF16 terms
    int *err = nullptr;  // set by a tensor-core kernel whose bounded wait expired
    mutable long problems[4] = {0, 0, 0, 0};   // GEMM problems per engine (SIMT, TMA, staged, BF16 sampling)
    mutable long timed = 0;                    // problems the engine tuner timed
};

// The fixed rule of tensor_cores = 1 / 2: long contractions only.  The
// Gauss-Jordan in-block updates (K = panel width <= 32) are memory bound per
// 128 x 128 tile and stay on FMA; the sampling products (K = |B|) and the
// K = 256 block-end updates of large fronts go to the tensor cores.
template <class T> bool use_tc(const Engine &e, const GemmDesc<T> &d) {
    return std::is_same<T, float>::value && e.tc != 0 && d.m >= 128 && d.n >= 32 && d.k >= 128;
}

enum { ENG_SIMT = 0, ENG_TMA = 1, ENG_STG = 2, ENG_BF16 = 3, NENG = 4 };

// ---- GEMM engine autotuner (tensor_cores = 3): per shape class (operand
// forms, sizes rounded up to powers of two) of the problems the TMA-fed
// tensor-core kernel can take, the first problem of the class is timed on the
// SIMT kernel and on that kernel, writing a scratch C; the tensor cores serve
// the class from then on when they were at least 15% faster (process-wide
// cache).  Other problems stay on SIMT.
struct EngChoice {
    int engine;
    float ms_simt, ms_tc;
};
static std::mutex g_eng_mu;
static std::unordered_map<uint64_t, EngChoice> g_eng_choice;
static std::vector<uint64_t> g_eng_order;   // keys in the order they were timed
static std::atomic<long> g_eng_timings{0};

static int ilog2c(long v) {
    int l = 0;
    while ((1L << l) < v) ++l;
    return l;
}

static uint64_t shape_key(const GemmDesc<float> &d, int tc_kind) {
    int dev = 0;
    cudaGetDevice(&dev);
    return ((uint64_t)dev << 48) | ((uint64_t)tc_kind << 40) | ((uint64_t)(d.transA != 0) << 39) |
           ((uint64_t)(d.B == nullptr) << 38) | ((uint64_t)ilog2c(d.m) << 24) | ((uint64_t)ilog2c(d.n) << 12) |
           (uint64_t)ilog2c(d.k);
}

// average time (ms) of two runs of problem d alone on engine `eng` after one warm-up run
static int time_engine(const Engine &E, const GemmDesc<float> &d, int eng, Work &W, cudaStream_t s, float *ms) {
    std::vector<GemmDesc<float>> dv{d};
    std::vector<GemmTile> tl;
    if (eng == ENG_SIMT) gemm_tiles_for(d, 0, tl);
    else gemm_tc_tiles_for(d, 0, tl);
    GemmDesc<float> *dd;
    GemmTile *dt;
    TmaGemmDesc *td = nullptr;
    int rc;
    if ((rc = W.up(dv, &dd)) || (rc = W.up(tl, &dt))) return rc;
    if (eng == ENG_TMA && (rc = gemm_tma_descs(dv, std::vector<char>{1}, W, &td))) return rc;
    auto launch = [&]() -> int {
        if (eng == ENG_SIMT) return gemm_batched<float>(dd, dt, (int)tl.size(), s, 0.0);
        if (eng == ENG_TMA) return gemm_tma(td, dt, (int)tl.size(), E.err, s, 0.0);
        return gemm_tc(dd, dt, (int)tl.size(), E.tc == 2 ? 0 : 1, E.err, s, 0.0);
    };
    cudaEvent_t e0, e1;
    HSS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "tuner events");
    }
    rc = launch();
    if (!rc) rc = cudaEventRecord(e0, s) == cudaSuccess ? HSS_OK : HSS_ECUDA;
    for (int r = 0; r < 2 && !rc; ++r) rc = launch();
    if (!rc) rc = cudaEventRecord(e1, s) == cudaSuccess ? HSS_OK : HSS_ECUDA;
    if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess ? HSS_OK : HSS_ECUDA;
    float t = 0.f;
    if (!rc) rc = cudaEventElapsedTime(&t, e0, e1) == cudaSuccess ? HSS_OK : HSS_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == HSS_ECUDA) return cuda_fail(cudaGetLastError(), "GEMM engine tuner");
    *ms = t / 2;
    return rc;
}

template <class T> int choose_engine(const Engine &E, const GemmDesc<T> &d, Work &W, cudaStream_t s, int *out) {
    *out = ENG_SIMT;
    if constexpr (std::is_same<T, float>::value) {
        // BF16 sampling: a precision choice of the FP32 form, for every sampling
        // product of at least one 128-row tile whose S the TMA can address
        if (E.bf16 && d.B == nullptr && d.m >= 128 && gemm_tma_eligible(d)) {
            *out = ENG_BF16;
            return HSS_OK;
        }
        if (E.tc == 0) return HSS_OK;
        const bool tma = gemm_tma_eligible(d);
        if (E.tc == 1 || E.tc == 2) {
            if (use_tc(E, d)) *out = (E.tc == 1 && tma) ? ENG_TMA : ENG_STG;
            return HSS_OK;
        }
        // tensor_cores = 3: chosen by timing, between SIMT and the TMA-fed kernel
        // (the thread-staging kernel lost to SIMT at every measured shape)
        if (d.m < 128 || d.n < 16 || d.k < 16 || !tma) return HSS_OK;
        const int tc = ENG_TMA;
        const uint64_t key = shape_key(d, tc);
        {
            std::lock_guard<std::mutex> lk(g_eng_mu);
            auto it = g_eng_choice.find(key);
            if (it != g_eng_choice.end()) {
                *out = it->second.engine;
                return HSS_OK;
            }
        }
        GemmDesc<float> t = d;   // same operands, masks and beta (the C traffic counts), a scratch C
        float *scratch;
        int rc;
        if ((rc = W.dalloc((size_t)d.m * d.n, &scratch))) return rc;
        HSS_CUDA(cudaMemsetAsync(scratch, 0, sizeof(float) * (size_t)d.m * d.n, s));
        t.C = scratch;
        t.ldc = d.m;
        float ms_simt = 0.f, ms_tc = 0.f;
        if ((rc = time_engine(E, t, ENG_SIMT, W, s, &ms_simt)) || (rc = time_engine(E, t, tc, W, s, &ms_tc))) return rc;
        g_eng_timings.fetch_add(1);
        E.timed++;
        // a clear margin: one problem alone on a warm L2 flatters the tensor-core kernel's
        // short launches a little against their place in a level-wide launch
        *out = ms_tc < 0.85f * ms_simt ? tc : ENG_SIMT;
        std::lock_guard<std::mutex> lk(g_eng_mu);
        if (!g_eng_choice.count(key)) g_eng_order.push_back(key);
        g_eng_choice[key] = EngChoice{*out, ms_simt, ms_tc};
    } else {
        (void)E;
        (void)d;
        (void)W;
        (void)s;
    }
    return HSS_OK;
}

// The GEMM launches of a stage: per launch group (a point of the kernel
// sequence), the tiles of its problems on each engine.
template <class T> struct GemmPlan {
    std::vector<GemmTile> tl[NENG];
    std::vector<int> off[NENG];
    std::vector<double> fl[NENG];
    TmaGemmDesc *d_tdescs = nullptr;
    GemmTile *d_tl[NENG] = {nullptr, nullptr, nullptr, nullptr};
};

// Engine of every problem, tiles per (group, engine), uploaded through W.
// Problems of a group keep their order.
template <class T>
int plan_gemms(const Engine &E, const std::vector<GemmDesc<T>> &descs, const std::vector<int> &group, int ngroups,
               GemmPlan<T> &P, Work &W, cudaStream_t s) {
    const size_t nd = descs.size();
    std::vector<int> which(nd, ENG_SIMT);
    std::vector<char> use_tma(nd, 0);
    int rc;
    for (size_t i = 0; i < nd; ++i) {
        if ((rc = choose_engine<T>(E, descs[i], W, s, &which[i]))) return rc;
        use_tma[i] = which[i] == ENG_TMA || which[i] == ENG_BF16;
        E.problems[which[i]]++;
    }
    std::vector<std::vector<int>> of(ngroups);
    for (size_t i = 0; i < nd; ++i) of[group[i]].push_back((int)i);
    for (int e = 0; e < NENG; ++e) {
        P.tl[e].clear();
        P.off[e].assign(ngroups + 1, 0);
        P.fl[e].assign(ngroups, 0.0);
    }
    for (int g = 0; g < ngroups; ++g) {
        for (int e = 0; e < NENG; ++e) P.off[e][g] = (int)P.tl[e].size();
        for (int i : of[g]) {
            const int e = which[i];
            if (e == ENG_SIMT) gemm_tiles_for(descs[i], i, P.tl[e]);
            else if constexpr (std::is_same<T, float>::value) gemm_tc_tiles_for(descs[i], i, P.tl[e]);
            P.fl[e][g] += gemm_flops(descs[i]);
        }
    }
    for (int e = 0; e < NENG; ++e) {
        P.off[e][ngroups] = (int)P.tl[e].size();
        if (!P.tl[e].empty() && (rc = W.up(P.tl[e], &P.d_tl[e]))) return rc;
    }
    if constexpr (std::is_same<T, float>::value) {
        // the tensor maps serve both TMA-fed kernels (TF32 split and BF16 sampling)
        if ((!P.tl[ENG_TMA].empty() || !P.tl[ENG_BF16].empty()) &&
            (rc = gemm_tma_descs(descs, use_tma, W, &P.d_tdescs)))
            return rc;
    }
    return HSS_OK;
}

// Launch group g of a plan: SIMT tiles, TMA tiles, staged tensor-core tiles
// (tma_class: the profile class of the TMA launches).
template <class T>
int run_gemm_group(const Engine &E, const GemmPlan<T> &P, const GemmDesc<T> *d_descs, int g, cudaStream_t s,
                   const char *tma_class = "gemm_tma") {
    int rc;
    for (int e = 0; e < NENG; ++e) {
        const int n = P.off[e][g + 1] - P.off[e][g];
        if (n <= 0) continue;
        const GemmTile *t = P.d_tl[e] + P.off[e][g];
        if (e == ENG_SIMT) {
            rc = gemm_batched<T>(d_descs, t, n, s, P.fl[e][g]);
        } else if constexpr (std::is_same<T, float>::value) {
            if ((e == ENG_TMA || e == ENG_BF16) && !P.d_tdescs) {
                set_error("GEMM plan: tensor-core tiles without tensor maps");
                return HSS_ECUDA;
            }
            if (e == ENG_TMA) rc = gemm_tma(P.d_tdescs, t, n, E.err, s, P.fl[e][g], tma_class);
            else if (e == ENG_BF16) rc = gemm_tma(P.d_tdescs, t, n, E.err, s, P.fl[e][g], "gemm_bf16_sample", true);
            else rc = gemm_tc(d_descs, t, n, E.tc == 2 ? 0 : 1, E.err, s, P.fl[e][g]);
        } else {
            rc = HSS_OK;
        }
        if (rc) return rc;
    }
    return HSS_OK;
}

template <class T> int choose_kb(int ni) {
    for (int kb = PANEL_KB_MAX; kb >= 8; kb /= 2)
        if ((long)ni * kb * (long)sizeof(T) + (long)ni * 4 <= PANEL_SMEM_MAX) return kb;
    return PANEL_KB_MAX;  // global-memory panel
}

// Blocked Gauss-Jordan sweep over the I pivots of every front of a stage.
// Per panel step: the panel kernels (register-resident where the panel fits,
// shared/global memory otherwise), the post-panel tiles, the trailing GEMM.
// pbeg/pend (HOST, per front, may be null): eliminate only the I columns
// [pbeg, pend), with pivots searched among the rows below pend -- one phase of
// an elimination split into phases (the structured merge; a phased sweep
// updates every column per panel, no blocking).
template <class T>
int eliminate_stage(const std::vector<FrontDev> &fr, const FrontDev *d_fr, T *arena, int *piv, int *rperm,
                    const int *ilist, int *iperm, int *status, double &exec_flops, const Engine &eng, Work &W,
                    cudaStream_t s, const int *pbeg = nullptr, const int *pend = nullptr) {
    HSS_HOST("eliminate_stage");
    int nf = (int)fr.size();
    const bool phased = pbeg != nullptr;
    std::vector<int> kb(nf), nsteps(nf), isreg(nf), Rf(nf), clpath(nf, 0), beg(nf), end(nf);
    std::vector<long> aoff(nf);
    long aold_total = 0;
    int maxsteps = 0;
    for (int f = 0; f < nf; ++f) {
        isreg[f] = 0;
        kb[f] = choose_kb<T>(fr[f].ni);
        for (int k = PANEL_KB_MAX; k >= 8; k /= 2)
            if (fr[f].ni > 0 && panel_reg_fits(k, fr[f].ni, (int)sizeof(T))) {
                kb[f] = k;
                isreg[f] = 1;
                break;
            }
        // tall fronts: 32-column panels spread over a cluster while their rows
        // exceed one CTA's registers, then the register panel
        if (fr[f].ni > PANEL_CL_MIN_NI && panel_cl_fits(PANEL_KB_MAX, fr[f].ni, (int)sizeof(T))) {
            kb[f] = PANEL_KB_MAX;
            clpath[f] = 1;
        }
        Rf[f] = cdiv(std::max(fr[f].ni, 1), PANEL_NT);
        beg[f] = phased ? pbeg[f] : 0;
        end[f] = phased ? pend[f] : fr[f].ni;
        nsteps[f] = end[f] > beg[f] ? cdiv(end[f] - beg[f], kb[f]) : 0;
        aoff[f] = aold_total;
        aold_total += (long)kb[f] * fr[f].n;
        maxsteps = std::max(maxsteps, nsteps[f]);
        exec_flops += 2.0 * fr[f].n * (double)fr[f].n * std::max(0, end[f] - beg[f]);
    }
    if (maxsteps == 0) return HSS_OK;
    struct Group {
        int off, cnt, reg, kb, rows;   // reg: 0 memory panel, 1 register panel, 2 cluster panel
        size_t smem;
        double flops;   // algorithmic work of the group's panels: 2 hT kb^2 each
    };
    // Large fronts (n >= PANEL_BLOCK_MIN_N) run in blocks of PANEL_BLOCK
    // panels: a panel's row moves and update reach only the columns of its
    // block; at the end of a block the other columns take the block's row
    // moves and one update of the block's width (for Gauss-Jordan,
    // C_out <- F(:, B) Aold(B, out) + C_out with the block's pivot rows
    // zeroed, the panel formula with B for the panel).  This reads the
    // trailing matrix once per block instead of once per panel, and the
    // K = 256 product suits the tensor cores; the cost is the explicit
    // inverse of the block's pivot rows in the update, whose rounding grows
    // with that block's condition, so smaller fronts keep per-panel updates.
    std::vector<long> aoffB(nf);
    long aoldB_total = 0;
    for (int f = 0; f < nf; ++f) {
        aoffB[f] = aoldB_total;
        aoldB_total += (long)PANEL_BLOCK * kb[f] * fr[f].n;
    }
    std::vector<PanelJob> jobs;
    std::vector<std::vector<int>> jobs_of(nf);
    std::vector<BlockJob> bjobs;
    std::vector<GemmDesc<T>> descs;
    std::vector<long> desc_b;        // offset of each descriptor's B operand in Aold (block: in AoldB)
    std::vector<char> desc_blk;
    std::vector<int> desc_group;     // launch group: 2 st (in-block update), 2 st + 1 (block end)
    std::vector<PanelTile> ptiles;
    std::vector<BlockTile> bptiles;
    std::vector<std::vector<Group>> groups(maxsteps);
    std::vector<int> ptile_off(maxsteps + 1), bptile_off(maxsteps + 1);
    long xtotal = 0, mtotal = 0;
    auto add_desc = [&](const GemmDesc<T> &d, long boff, bool blk, int grp) {
        descs.push_back(d);
        desc_b.push_back(boff);
        desc_blk.push_back(blk);
        desc_group.push_back(grp);
    };
    for (int st = 0; st < maxsteps; ++st) {
        ptile_off[st] = (int)ptiles.size();
        bptile_off[st] = (int)bptiles.size();
        std::vector<int> act;
        for (int f = 0; f < nf; ++f)
            if (st < nsteps[f]) act.push_back(f);
        // panel kind of this step: register (isreg, or a cluster-path front whose
        // rows now fit one CTA), cluster, memory
        auto hT_at = [&](int f) { return fr[f].ni - (beg[f] + st * kb[f]); };
        auto kind = [&](int f) {
            if (isreg[f]) return 1;
            if (!clpath[f]) return 0;
            return panel_reg_fits(kb[f], hT_at(f), (int)sizeof(T)) ? 1 : 2;
        };
        // register panels grouped by (kb, rows of this step's variant), then the
        // memory panels; the variant follows the rows left at this step
        auto step_rows = [&](int f) {
            const int hTs = hT_at(f);
            if (hTs <= PANEL_SMALL_NT) return PANEL_SMALL_NT;
            if (hTs <= 2 * PANEL_SMALL_NT) return 2 * PANEL_SMALL_NT;
            return cdiv(hTs, PANEL_NT) * PANEL_NT;
        };
        auto group_rows = [&](int f) {
            const int k = kind(f);
            if (k == 1) return step_rows(f);
            if (k == 2) return panel_cl_capacity(hT_at(f), (int)sizeof(T));
            return Rf[f] * PANEL_NT;
        };
        std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
            if (kind(a) != kind(b)) return kind(a) > kind(b);
            if (kb[a] != kb[b]) return kb[a] < kb[b];
            return group_rows(a) < group_rows(b);
        });
        for (int f : act) {
            const int n = fr[f].n;
            int k0 = beg[f] + st * kb[f];
            int kbs = std::min(kb[f], end[f] - k0);
            // fronts below PANEL_BLOCK_MIN_N (and phased sweeps): one block
            // spanning every column (the plain per-panel update)
            const bool blocked = n >= PANEL_BLOCK_MIN_N && !phased;
            const int K0 = blocked ? (st / PANEL_BLOCK) * PANEL_BLOCK * kb[f] : 0;
            const int bw = blocked ? std::min(PANEL_BLOCK * kb[f], fr[f].ni - K0) : n;
            size_t hT = (size_t)(fr[f].ni - k0);
            int use_smem = 0;
            size_t need = 0;
            const int knd = kind(f);
            if (knd != 0) {
                use_smem = 2;
                need = 3 * hT * sizeof(int);
            } else {
                need = hT * kbs * sizeof(T) + hT * sizeof(int);
                use_smem = need <= (size_t)PANEL_SMEM_MAX;
                if (!use_smem) need = hT * sizeof(int);
            }
            auto &gs = groups[st];
            if (gs.empty() || gs.back().reg != knd ||
                (knd != 0 && (gs.back().kb != kb[f] || gs.back().rows != group_rows(f))))
                gs.push_back({(int)jobs.size(), 0, knd, kb[f], group_rows(f), 0, 0.0});
            gs.back().cnt++;
            gs.back().flops += 2.0 * (double)hT * kbs * kbs;
            gs.back().smem = std::max(gs.back().smem, need);
            int jid = (int)jobs.size();
            jobs.push_back({f, k0, kbs, end[f], use_smem, aoff[f], xtotal, mtotal});
            jobs_of[f].push_back(jid);
            xtotal += (long)kbs * kbs;
            mtotal += 1 + 4 * PANEL_KB_MAX;
            // in-block columns [K0, K0 + bw) outside the panel
            for (int c0 = K0; c0 < K0 + bw; c0 += 32)
                if (!(c0 >= k0 && c0 + 32 <= k0 + kbs)) ptiles.push_back({jid, 0, c0, K0, K0 + bw});
            int nout = n - (fr[f].ni - k0);
            for (int r0 = 0; r0 < nout; r0 += 64) ptiles.push_back({jid, 1, r0, 0, 0});
            GemmDesc<T> d{};
            d.A = arena + fr[f].foff + (long)n * k0;
            d.lda = n;
            d.B = nullptr;  // Aold of this job (columns from K0), set once the workspace exists
            d.C = arena + fr[f].foff + (long)n * K0;
            d.ldc = n;
            d.ldb = kbs;
            d.m = n;
            d.n = bw;
            d.k = kbs;
            d.transA = 0;
            d.transB = 0;
            d.alpha = T(1);
            d.beta = T(1);
            d.zr_lo = k0;
            d.zr_hi = k0 + kbs;
            d.skip_lo = k0 - K0;
            d.skip_hi = k0 - K0 + kbs;
            if (bw > kbs) add_desc(d, aoff[f] + (long)kbs * K0, false, 2 * st);
            // end of the block: the other columns
            const bool block_end = blocked && ((st % PANEL_BLOCK == PANEL_BLOCK - 1) || st == nsteps[f] - 1);
            if (block_end && n > bw) {
                BlockJob bj{};
                bj.front = f;
                bj.k0 = K0;
                bj.width = bw;
                bj.np = st % PANEL_BLOCK + 1;
                for (int q = 0; q < bj.np; ++q) bj.job[q] = jobs_of[f][st - bj.np + 1 + q];
                bj.aoff = aoffB[f];
                const int bjid = (int)bjobs.size();
                bjobs.push_back(bj);
                for (int c0 = 0; c0 < n; c0 += 32)
                    if (!(c0 >= K0 && c0 + 32 <= K0 + bw)) bptiles.push_back({bjid, c0});
                GemmDesc<T> e{};
                e.A = arena + fr[f].foff + (long)n * K0;
                e.lda = n;
                e.B = nullptr;   // AoldB, set once the workspace exists
                e.ldb = bw;
                e.C = arena + fr[f].foff;
                e.ldc = n;
                e.m = n;
                e.n = n;
                e.k = bw;
                e.transA = 0;
                e.transB = 0;
                e.alpha = T(1);
                e.beta = T(1);
                e.zr_lo = K0;
                e.zr_hi = K0 + bw;
                e.skip_lo = K0;
                e.skip_hi = K0 + bw;
                add_desc(e, aoffB[f], true, 2 * st + 1);
            }
        }
    }
    ptile_off[maxsteps] = (int)ptiles.size();
    bptile_off[maxsteps] = (int)bptiles.size();
    T *d_aold, *d_aoldB, *d_x;
    int *d_mv;
    PanelJob *d_jobs;
    BlockJob *d_bjobs;
    GemmDesc<T> *d_descs;
    PanelTile *d_ptiles;
    BlockTile *d_bptiles;
    int rc;
    if ((rc = W.dalloc(aold_total, &d_aold)) || (rc = W.dalloc(std::max(aoldB_total, 1L), &d_aoldB)) ||
        (rc = W.dalloc(xtotal, &d_x)) || (rc = W.dalloc(mtotal, &d_mv)))
        return rc;
    for (size_t i = 0; i < descs.size(); ++i) descs[i].B = (desc_blk[i] ? d_aoldB : d_aold) + desc_b[i];
    GemmPlan<T> plan;
    {
        HSS_HOST("eliminate_upload_plan");
        if ((rc = W.up(jobs, &d_jobs)) || (rc = W.up(bjobs, &d_bjobs)) || (rc = W.up(descs, &d_descs)) ||
            (rc = W.up(ptiles, &d_ptiles)) || (rc = W.up(bptiles, &d_bptiles)) ||
            (rc = plan_gemms<T>(eng, descs, desc_group, 2 * maxsteps, plan, W, s)))
            return rc;
    }
    HSS_HOST("eliminate_launch");
    for (int st = 0; st < maxsteps; ++st) {
        for (const Group &g : groups[st]) {
            if (g.reg == 1)
                rc = launch_gj_panel_reg<T>(d_jobs + g.off, g.cnt, g.kb, g.rows, d_fr, arena, d_x, d_mv, piv, rperm,
                                            ilist, iperm, status, s, g.flops);
            else if (g.reg == 2)
                rc = launch_gj_panel_cl<T>(d_jobs + g.off, g.cnt, g.rows, g.smem, d_fr, arena, d_x, d_mv, piv, rperm,
                                           ilist, iperm, status, s, g.flops);
            else
                rc = launch_gj_panel<T>(d_jobs + g.off, g.cnt, g.smem, d_fr, arena, d_x, d_mv, piv, rperm, ilist,
                                        iperm, status, s, g.flops);
            if (rc) return rc;
        }
        if ((rc = launch_gj_post<T>(d_ptiles + ptile_off[st], ptile_off[st + 1] - ptile_off[st], d_jobs, d_fr, arena,
                                    d_aold, d_x, d_mv, s)))
            return rc;
        if ((rc = run_gemm_group<T>(eng, plan, d_descs, 2 * st, s, "gemm_tma_update"))) return rc;
        if ((rc = launch_gj_block_post<T>(d_bptiles + bptile_off[st], bptile_off[st + 1] - bptile_off[st], d_bjobs,
                                          d_jobs, d_fr, arena, d_aoldB, d_mv, s)))
            return rc;
        if ((rc = run_gemm_group<T>(eng, plan, d_descs, 2 * st + 1, s, "gemm_tma_block"))) return rc;
    }
    return HSS_OK;
}

struct RoundFront {     // a front of the current sampling round
    int f;              // stage-local front
    int r;
};

// Blocks compressed that are not a box's Schur complement (the structured
// merge's second Schur complement S~ of a parent's interior block, Algorithm 1
// step 2.2): per front its HSS nodes, its test-matrix counter key and the map
// of its rows to positions in the target front (DEVICE); these take r0 as
// their first width and no residual probe, and leave no log record.
struct CompressOverride {
    std::vector<const std::vector<HssNode> *> nodes;
    std::vector<int> key;
    std::vector<const int *> fmap;
};

// Randomized HSS compression of the stage's Schur complements, written into
// the parent fronts.  Fronts whose HSS tree is a single node (or with
// compression off) copy S unchanged.  With `ov`, the blocks of `ov` instead.
template <class T>
int compress_stage(const hss_tree *t, const hss_factor_opts &o, const std::vector<FrontDev> &fr,
                   const std::vector<int> &boxes, const std::vector<long> &poff, const std::vector<int> &pn,
                   const std::vector<long> &keep_h, T *arena, T *keep, int *status_dev, int nstatus,
                   std::vector<FrontLog> &logv, hss_factor_t *F, const Engine &eng, Work &W, cudaStream_t s,
                   const CompressOverride *ov = nullptr) {
    HSS_HOST("compress_stage");
    int nf = (int)fr.size();
    int rc;
    auto nodes_of = [&](int f) -> const std::vector<HssNode> & { return ov ? *ov->nodes[f] : t->hss[boxes[f]]; };
    auto key_of = [&](int f) { return ov ? ov->key[f] : t->box_local[boxes[f]]; };
    std::vector<ExpandFront> ef(nf);
    for (int f = 0; f < nf; ++f) {
        const FrontDev &d = fr[f];
        ef[f].S = arena + d.foff + d.ni + (long)d.n * d.ni;
        ef[f].lds = d.n;
        ef[f].nb = d.nb;
        ef[f].fmap = ov ? ov->fmap[f] : t->d_fmap.as<int>() + t->boff[boxes[f]];
        ef[f].poff = poff[f];
        ef[f].pn = pn[f];
        ef[f].keep_h = keep_h[f];
    }
    ExpandFront *d_ef;
    if ((rc = W.up(ef, &d_ef))) return rc;

    std::vector<RoundFront> active;
    std::vector<ExpandItem> plain_items;
    std::vector<int> rounds(nf, 0), kmax(nf, 0), rfin(nf, 0);
    std::vector<char> capped(nf, 0);
    for (int f = 0; f < nf; ++f) {
        int b = boxes[f];
        if (fr[f].nb == 0) continue;
        bool comp = o.compress && nodes_of(f).size() > 1;
        if (comp) {
            const int r_first = (o.r_init && !ov) ? std::max(1, std::min(o.r_init[b], o.rmax)) : std::min(o.r0, o.rmax);
            active.push_back({f, r_first});
        } else {
            for (int r0 = 0; r0 < fr[f].nb; r0 += EXP_TILE)
                for (int c0 = 0; c0 < fr[f].nb; c0 += EXP_TILE)
                    plain_items.push_back({0, f, -1, -1, r0, c0, 0, fr[f].nb, 0, fr[f].nb});
        }
    }
    if (!plain_items.empty()) {
        ExpandItem *d_items;
        if ((rc = W.up(plain_items, &d_items))) return rc;
        if ((rc = launch_hss_expand<T>(d_items, (int)plain_items.size(), nullptr, nullptr, d_ef, nullptr, nullptr,
                                       arena, keep, 0, s)))
            return rc;
    }

    while (!active.empty()) {
        int nc = (int)active.size();
        HSS_HOST("compress_round");
        // ---- node table, workspace layout
        std::vector<CompFront<T>> cfs(nc);
        std::vector<NodeDev> nodes;
        std::vector<int> node_base(nc + 1);
        long wsz = 0, isz = 0;
        for (int c = 0; c < nc; ++c) {
            const FrontDev &d = fr[active[c].f];
            int r = active[c].r;
            cfs[c].S = arena + d.foff + d.ni + (long)d.n * d.ni;
            cfs[c].lds = d.n;
            cfs[c].nb = d.nb;
            cfs[c].r = r;
            cfs[c].box = key_of(active[c].f);
            cfs[c].yoff = wsz;
            wsz += (long)d.nb * r;
            cfs[c].zoff = wsz;
            wsz += (long)d.nb * r;
            const auto &hn = nodes_of(active[c].f);
            node_base[c] = (int)nodes.size();
            int root = (int)hn.size() - 1;
            for (int i = 0; i < (int)hn.size(); ++i) {
                NodeDev nd{};
                nd.cf = c;
                nd.lo = hn[i].lo;
                nd.hi = hn[i].hi;
                nd.a = hn[i].a >= 0 ? node_base[c] + hn[i].a : -1;
                nd.b = hn[i].b >= 0 ? node_base[c] + hn[i].b : -1;
                int mcap = nd.a < 0 ? hn[i].hi - hn[i].lo
                                    : nodes[nd.a].s[0].kcap + nodes[nd.b].s[0].kcap;
                int kcap = std::min(mcap, r);
                for (int sd = 0; sd < 2; ++sd) {
                    NodeSide &ns = nd.s[sd];
                    ns.mcap = mcap;
                    ns.kcap = kcap;
                    if (i == root) continue;
                    ns.loff = wsz; wsz += (long)mcap * r;
                    ns.toff = wsz; wsz += (long)kcap * mcap;
                    ns.skoff = wsz; wsz += (long)kcap * r;
                    ns.tloff = wsz; wsz += (long)kcap * r;
                    ns.talloff = wsz; wsz += (long)(hn[i].hi - hn[i].lo) * kcap;
                    ns.ordoff = isz; isz += mcap;
                    ns.skioff = isz; isz += kcap;
                }
                nodes.push_back(nd);
            }
        }
        node_base[nc] = (int)nodes.size();
        int nn = (int)nodes.size();
        T *ws;
        int *d_iws, *d_kout, *d_fk;
        NodeDev *d_nodes;
        CompFront<T> *d_cfs;
        if ((rc = W.dalloc(wsz, &ws)) || (rc = W.dalloc(isz, &d_iws)) || (rc = W.up(nodes, &d_nodes)) ||
            (rc = W.up(cfs, &d_cfs)) || (rc = W.dalloc(2 * nn, &d_kout)) || (rc = W.dalloc(nc, &d_fk)))
            return rc;
        HSS_CUDA(cudaMemsetAsync(d_kout, 0, sizeof(int) * 2 * nn, s));
        HSS_CUDA(cudaMemsetAsync(d_fk, 0, sizeof(int) * nc, s));
        // ---- sampling Y = S Omega, Z = S^t Psi, then the leaf corrections
        std::vector<GemmDesc<T>> g1, g2;
        std::vector<GemmTile> t2;   // leaf corrections (SIMT)
        for (int c = 0; c < nc; ++c) {
            GemmDesc<T> d{};
            d.A = cfs[c].S;
            d.lda = (int)cfs[c].lds;
            d.B = nullptr;
            d.m = cfs[c].nb;
            d.n = cfs[c].r;
            d.k = cfs[c].nb;
            d.alpha = T(1);
            d.beta = T(0);
            d.zr_lo = d.zr_hi = 0;
            d.skip_lo = d.skip_hi = 0;
            d.seed = o.seed;
            d.front = cfs[c].box;
            d.brow0 = 0;
            d.ldc = cfs[c].nb;
            d.C = ws + cfs[c].yoff;
            d.transA = 0;
            d.stream = 0;
            g1.push_back(d);
            d.C = ws + cfs[c].zoff;
            d.transA = 1;
            d.stream = 1;
            g1.push_back(d);
            for (int i = node_base[c]; i < node_base[c + 1]; ++i) {
                if (nodes[i].a >= 0) continue;
                int lo = nodes[i].lo, m = nodes[i].hi - nodes[i].lo;
                GemmDesc<T> e = d;
                e.A = cfs[c].S + lo + cfs[c].lds * lo;
                e.m = m;
                e.k = m;
                e.alpha = T(-1);
                e.beta = T(1);
                e.brow0 = lo;
                e.C = ws + cfs[c].yoff + lo;
                e.transA = 0;
                e.stream = 0;
                g2.push_back(e);
                gemm_tiles_for(g2.back(), (int)g2.size() - 1, t2);
                e.C = ws + cfs[c].zoff + lo;
                e.transA = 1;
                e.stream = 1;
                g2.push_back(e);
                gemm_tiles_for(g2.back(), (int)g2.size() - 1, t2);
            }
        }
        {
            HSS_HOST("compress_sample");
            GemmDesc<T> *a, *c2;
            GemmTile *d2;
            GemmPlan<T> plan;
            if ((rc = W.up(g1, &a)) || (rc = W.up(g2, &c2)) || (rc = W.up(t2, &d2)) ||
                (rc = plan_gemms<T>(eng, g1, std::vector<int>(g1.size(), 0), 1, plan, W, s)))
                return rc;
            double f2 = 0;
            for (auto &d : g2) f2 += gemm_flops(d);
            if ((rc = run_gemm_group<T>(eng, plan, a, 0, s, "gemm_tma_sample"))) return rc;
            if ((rc = gemm_batched<T>(c2, d2, (int)t2.size(), s, f2))) return rc;
        }
        // ---- interpolative decompositions, deepest HSS level first
        HSS_HOST("compress_id_decide_expand");
        int maxd = 0;
        std::vector<int> ndepth(nn, 0);
        for (int c = 0; c < nc; ++c) {
            const auto &hn = nodes_of(active[c].f);
            for (int i = 0; i < (int)hn.size(); ++i) {
                ndepth[node_base[c] + i] = hn[i].depth;
                maxd = std::max(maxd, hn[i].depth);
            }
        }
        std::vector<std::vector<int>> work(maxd + 1);
        std::vector<size_t> idsmem(maxd + 1, 0), tallsmem(maxd + 1, 0);
        for (int i = 0; i < nn; ++i) {
            int dpt = ndepth[i];
            if (dpt == 0) continue;  // roots carry no basis
            int r = cfs[nodes[i].cf].r;
            int mcap = nodes[i].s[0].mcap, kcap = nodes[i].s[0].kcap;
            work[dpt].push_back(2 * i);
            work[dpt].push_back(2 * i + 1);
            idsmem[dpt] = std::max(idsmem[dpt], id_smem_bytes(r, mcap, (int)sizeof(T)));
            tallsmem[dpt] = std::max(tallsmem[dpt], sizeof(int) * (mcap + 2) + sizeof(T) * (size_t)mcap * kcap + 16);
        }
        for (int dpt = maxd; dpt >= 1; --dpt) {
            if (work[dpt].empty()) continue;
            int *d_work;
            if ((rc = W.up(work[dpt], &d_work))) return rc;
            if ((rc = launch_hss_id<T>(d_nodes, d_work, (int)work[dpt].size(), d_cfs, ws, d_iws, d_kout, d_fk,
                                       (T)o.tol, o.seed, idsmem[dpt], s)))
                return rc;
        }
        std::vector<int> hfk(nc);
        if ((rc = factor_readback(hfk.data(), d_fk, sizeof(int) * nc, s, F))) return rc;
        // ---- decide: fronts whose rank reached r - oversample sample again, wider
        // A front whose rank still needs more samples when the cap rmax stops
        // the growth has no oversampling margin left: Theorem 1's error bound
        // (l = k + p samples) does not hold, so it keeps S itself (H = S), or,
        // under HSS_CAP_ACCEPT, the approximant from the r samples it has (the
        // IDs already allow ranks up to r).
        std::vector<RoundFront> next;
        std::vector<char> done(nc, 0), dense(nc, 0);
        for (int c = 0; c < nc; ++c) {
            int f = active[c].f, r = active[c].r;
            rounds[f]++;
            kmax[f] = hfk[c];
            rfin[f] = r;
            const bool short_of_samples = hfk[c] > r - o.oversample && r < fr[f].nb;
            if (short_of_samples && r + o.dr <= o.rmax) {
                next.push_back({f, r + o.dr});
            } else {
                done[c] = 1;
                dense[c] = short_of_samples && o.cap_policy == HSS_CAP_KEEP;
                capped[f] = short_of_samples;
            }
        }
        // ---- expansion of the finished fronts: tall bases, then H tiles
        for (int dpt = maxd; dpt >= 1; --dpt) {
            std::vector<int> wk;
            for (int x : work[dpt])
                if (done[nodes[x >> 1].cf] && !dense[nodes[x >> 1].cf]) wk.push_back(x);
            if (wk.empty()) continue;
            int *d_wk;
            if ((rc = W.up(wk, &d_wk))) return rc;
            if ((rc = launch_hss_tall<T>(d_nodes, d_wk, (int)wk.size(), d_kout, ws, d_iws, tallsmem[dpt], s)))
                return rc;
        }
        std::vector<ExpandItem> items;
        int kmax_done = 0;
        for (int c = 0; c < nc; ++c) {
            if (!done[c]) continue;
            int f = active[c].f;
            if (dense[c]) {
                for (int r0 = 0; r0 < fr[f].nb; r0 += EXP_TILE)
                    for (int c0 = 0; c0 < fr[f].nb; c0 += EXP_TILE)
                        items.push_back({0, f, -1, -1, r0, c0, 0, fr[f].nb, 0, fr[f].nb});
                continue;
            }
            kmax_done = std::max(kmax_done, hfk[c]);
            for (int i = node_base[c]; i < node_base[c + 1]; ++i) {
                const NodeDev &N = nodes[i];
                if (N.a < 0) {
                    for (int r0 = N.lo; r0 < N.hi; r0 += EXP_TILE)
                        for (int c0 = N.lo; c0 < N.hi; c0 += EXP_TILE)
                            items.push_back({0, f, -1, -1, r0, c0, N.lo, N.hi, N.lo, N.hi});
                    continue;
                }
                const NodeDev &Na = nodes[N.a], &Nb = nodes[N.b];
                for (int pass = 0; pass < 2; ++pass) {
                    int x = pass ? N.b : N.a, y = pass ? N.a : N.b;
                    const NodeDev &X = pass ? Nb : Na, &Y = pass ? Na : Nb;
                    for (int r0 = X.lo; r0 < X.hi; r0 += EXP_TILE)
                        for (int c0 = Y.lo; c0 < Y.hi; c0 += EXP_TILE)
                            items.push_back({1, f, x, y, r0, c0, X.lo, X.hi, Y.lo, Y.hi});
                }
            }
        }
        if (!items.empty()) {
            ExpandItem *d_items;
            if ((rc = W.up(items, &d_items))) return rc;
            if ((rc = launch_hss_expand<T>(d_items, (int)items.size(), d_nodes, d_kout, d_ef, ws, d_iws, arena, keep,
                                           kmax_done, s)))
                return rc;
        }
        // ---- residual probe of the approximants accepted in this sampling round: a front
        // with ||(S - H) W|| > 10 tol depth ||S W|| samples again with r + dr
        if (o.probe > 0 && !ov) {
            std::vector<ProbeItem> pit;
            std::vector<ProbeFront> pfr;
            std::vector<int> pc;   // round-front index of each probed front
            long rows = 0;   // doubles of row sums: per front, column tiles x rows x 2 PROBE_MAX
            for (int c = 0; c < nc; ++c) {
                if (!done[c] || dense[c]) continue;
                const int f = active[c].f, slot = (int)pc.size();
                const long ra = rows;
                pc.push_back(c);
                pfr.push_back({f, ra});
                rows += (long)cdiv(fr[f].nb, PROBE_NT) * fr[f].nb * 2 * PROBE_MAX;
                for (int r0 = 0; r0 < fr[f].nb; r0 += PROBE_NT)
                    for (int c0 = 0; c0 < fr[f].nb; c0 += PROBE_NT)
                        pit.push_back({slot, f, t->box_local[boxes[f]], r0, c0, ra});
            }
            if (!pit.empty()) {
                ProbeItem *d_pit;
                ProbeFront *d_pfr;
                double *d_acc, *d_rowacc;
                if ((rc = W.up(pit, &d_pit)) || (rc = W.up(pfr, &d_pfr)) || (rc = W.dalloc(2 * pc.size(), &d_acc)) ||
                    (rc = W.dalloc((size_t)rows, &d_rowacc)))
                    return rc;
                if ((rc = launch_hss_probe<T>(d_pit, (int)pit.size(), d_pfr, (int)pfr.size(), d_ef, arena, o.seed,
                                              o.probe, d_rowacc, d_acc, s)))
                    return rc;
                std::vector<double> acc(2 * pc.size());
                if ((rc = factor_readback(acc.data(), d_acc, sizeof(double) * acc.size(), s, F))) return rc;
                for (size_t k = 0; k < pc.size(); ++k) {
                    const int f = active[pc[k]].f, r = active[pc[k]].r;
                    int depth = 1;
                    for (const auto &hn : t->hss[boxes[f]]) depth = std::max(depth, hn.depth);
                    const double rel = acc[2 * k + 1] > 0 ? std::sqrt(acc[2 * k] / acc[2 * k + 1]) : 0.0;
                    if (rel > 10.0 * o.tol * depth && r + o.dr <= o.rmax && r < fr[f].nb) {
                        next.push_back({f, r + o.dr});
                        F->probe_regrown++;
                    }
                }
            }
        }
        active.swap(next);
    }
    for (int f = 0; f < nf; ++f) {
        if (ov) {   // blocks of the structured merge: no log record, the widths and ranks still counted
            F->max_rank = std::max(F->max_rank, kmax[f]);
            F->max_r = std::max(F->max_r, rfin[f]);
            continue;
        }
        int b = boxes[f];
        FrontLog lg{b, t->level[b], fr[f].ni, fr[f].nb, rfin[f], rounds[f], kmax[f], (int)t->hss[b].size()};
        logv.push_back(lg);
        F->max_rank = std::max(F->max_rank, kmax[f]);
        F->max_r = std::max(F->max_r, rfin[f]);
        F->rounds = std::max(F->rounds, rounds[f]);
        F->capped_fronts += capped[f];
    }
    (void)status_dev;
    (void)nstatus;
    return HSS_OK;
}

// Fronts and byte counts of one apply stage (its work items are built by
// pack_apply once every stage exists).
static void build_apply_stage(ApplyStage &as, const std::vector<FrontDev> &fr, bool top) {
    as.top = top;
    as.nfronts = (int)fr.size();
    as.h_fronts = fr;
    as.fwd_bytes = as.bwd_bytes = as.fwd_vec = as.bwd_vec = 0;
    for (int f = 0; f < (int)fr.size(); ++f) {
        if (fr[f].ni == 0) continue;
        as.fwd_bytes += 8.0 * fr[f].n * (double)fr[f].ni;
        as.bwd_bytes += 8.0 * fr[f].ni * (double)fr[f].nb;
        as.fwd_vec += fr[f].ni + fr[f].ni + 2.0 * fr[f].nb;      // x_I read, t written, x_B read+written
        as.bwd_vec += fr[f].nb + fr[f].ni + fr[f].ni;           // x_B read, t read, x_I written
    }
}

// The structured merge (reading R2: eq. (37), Algorithm 1 step 2, Algorithm 3)
// on dense fronts.  The interior of a parent front is [B^mu n I ; B^nu n I]
// (n1 rows from the first child).  Phase 1 eliminates the first n1 pivots with
// pivots searched among those rows only, which leaves the second Schur
// complement S~ = S2 - A21 S1^-1 A12 in the trailing interior block; S~ is
// replaced there by its HSS approximant H~ (Theorem 1, its own tree and test
// matrices); phase 2 eliminates the remaining pivots.  The result is the
// Gauss-Jordan factorization of the front with A_ii + blockdiag(0, H~ - S~) in
// place of A_ii, whose inverse is eq. (37)'s block solve, so W, S and the
// stored blocks the apply uses are those of R2.
template <class T>
int eliminate_structured(const hss_tree *t, const hss_factor_opts &o, const std::vector<FrontDev> &fr,
                         const FrontDev *d_fr, const std::vector<int> &n1, const std::vector<std::vector<int>> &dofs2,
                         const std::vector<int> &tree_box, const std::vector<int> &key,
                         const std::vector<int> &hss_of_box, T *arena, int *piv, int *rperm, const int *ilist,
                         int *iperm, int *status, double &exec_flops, hss_factor_t *F, const Engine &eng, Work &W,
                         cudaStream_t s) {
    const int nf = (int)fr.size();
    std::vector<int> zero(nf, 0), ni(nf);
    for (int f = 0; f < nf; ++f) ni[f] = fr[f].ni;
    int rc;
    if ((rc = eliminate_stage<T>(fr, d_fr, arena, piv, rperm, ilist, iperm, status, exec_flops, eng, W, s, zero.data(),
                                 n1.data())))
        return rc;
    // S~ blocks: one pseudo-front per front with a trailing interior block
    std::vector<FrontDev> sv;
    std::vector<int> svbox;
    std::vector<long> poff, keeph;
    std::vector<int> pn;
    CompressOverride ov;
    std::vector<std::vector<HssNode>> nodes_store(nf);
    std::vector<int> fmap_all;
    std::vector<long> fmap_off;
    const std::vector<int> elem_pos = elem_positions(t);
    for (int f = 0; f < nf; ++f) {
        const int m2 = fr[f].ni - n1[f];
        if (m2 <= 0) continue;
        FrontDev d{};
        d.foff = fr[f].foff + n1[f] + (long)fr[f].n * n1[f];
        d.n = fr[f].n;   // leading dimension
        d.ni = 0;
        d.nb = m2;
        d.box = fr[f].box;
        sv.push_back(d);
        svbox.push_back(fr[f].box >= 0 ? fr[f].box : 0);
        poff.push_back(fr[f].foff);
        pn.push_back(fr[f].n);
        keeph.push_back(-1);
        if (hss_of_box[f] >= 0) {
            ov.nodes.push_back(&t->hss[hss_of_box[f]]);
        } else {
            hss_nodes_over(t, elem_pos, tree_box[f], dofs2[f], nodes_store[f]);
            ov.nodes.push_back(&nodes_store[f]);
        }
        ov.key.push_back(key[f]);
        fmap_off.push_back((long)fmap_all.size());
        for (int i = 0; i < m2; ++i) fmap_all.push_back(n1[f] + i);   // in place: H~ over S~
    }
    if (!sv.empty()) {
        int *d_fmap;
        if ((rc = W.up(fmap_all, &d_fmap))) return rc;
        for (long off : fmap_off) ov.fmap.push_back(d_fmap + off);
        std::vector<FrontLog> nolog;
        if ((rc = compress_stage<T>(t, o, sv, svbox, poff, pn, keeph, arena, (T *)nullptr, nullptr, 0, nolog, F, eng,
                                    W, s, &ov)))
            return rc;
    }
    return eliminate_stage<T>(fr, d_fr, arena, piv, rperm, ilist, iperm, status, exec_flops, eng, W, s, n1.data(),
                              ni.data());
}

template <class T> int factor_impl(const hss_bsr *A, const hss_tree *t, const hss_factor_opts &o, cudaStream_t s,
                                   hss_factor_t *F) {
    const int nbox = t->nbox;
    int rc;
    std::vector<long> foff(nbox);
    long total = 0;
    for (int b = 0; b < nbox; ++b) {
        long n = t->ni[b] + t->nb[b];
        foff[b] = total;
        total += (n * n + 31) / 32 * 32;
    }
    // one top block A^(0) per instance (a plain tree is a forest of one)
    const int ninst = t->ninst;
    std::vector<int> ntop_i(ninst), top_off(ninst + 1, 0);
    std::vector<long> foff_top(ninst);
    std::vector<int> topset;
    for (int i = 0; i < ninst; ++i) {
        const int b0 = t->inst_top[i];
        ntop_i[i] = t->nb[b0] + t->nb[b0 + 1];
        foff_top[i] = total;
        total += ((long)ntop_i[i] * ntop_i[i] + 31) / 32 * 32;
        top_off[i + 1] = top_off[i] + ntop_i[i];
        topset.insert(topset.end(), t->bset.begin() + t->boff[b0], t->bset.begin() + t->boff[b0 + 2]);
    }
    const int ntop = top_off[ninst];
    F->ntop = ntop;
    if ((rc = F->arena.alloc(sizeof(T) * std::max(total, 1L)))) return rc;
    HSS_CUDA(cudaMemsetAsync(F->arena.p, 0, sizeof(T) * total, s));
    T *arena = F->arena_ptr<T>();
    const int ilen = t->ioff[nbox];
    const bool structured = o.merge == 1 && o.compress;
    Work WL(s);   // scratch for the whole call (never reset)
    ScratchPtr d_piv, d_scratch, d_slot, d_tcerr;
    if ((rc = upload(F->d_topset, topset, s)) || (rc = F->d_iperm.alloc(sizeof(int) * (ilen + ntop + 1))) ||
        (rc = WL.dalloc_bytes(sizeof(int) * (ilen + ntop + 1), &d_piv.p)) ||
        (rc = WL.dalloc_bytes(sizeof(int) * (ilen + ntop + 1), &d_scratch.p)) ||
        (rc = WL.dalloc_bytes(sizeof(int) * t->nelem, &d_slot.p)) || (rc = WL.dalloc_bytes(sizeof(int), &d_tcerr.p)))
        return rc;
    HSS_CUDA(cudaMemsetAsync(d_slot.p, 0xff, sizeof(int) * t->nelem, s));
    // optional copies of S and H
    F->keep_s.assign(nbox, -1);
    F->keep_h.assign(nbox, -1);
    if (o.keep_schur) {
        long ks = 0;
        for (int b = 0; b < nbox; ++b) {
            F->keep_s[b] = ks;
            ks += (long)t->nb[b] * t->nb[b];
            F->keep_h[b] = ks;
            ks += (long)t->nb[b] * t->nb[b];
        }
        if ((rc = F->keep.alloc(sizeof(T) * std::max(ks, 1L)))) return rc;
    }
    T *keep = F->keep.as<T>();
    // zero-pivot flags of every front of every stage and of the top blocks,
    // read once at the end of the call
    // (one more flag after them: a NaN or infinite value in A)
    size_t nstat = (size_t)ninst;
    for (const auto &st : t->stages) nstat += st.size();
    ScratchPtr d_status_all;
    if ((rc = WL.dalloc_bytes(sizeof(int) * (nstat + 1), &d_status_all.p))) return rc;
    HSS_CUDA(cudaMemsetAsync(d_status_all.p, 0, sizeof(int) * (nstat + 1), s));
    {
        HSS_PROF("check_finite", s);
        k_check_finite<<<2 * device_sms(), 256, 0, s>>>(A->row_ptr, A->nb, A->bs * A->bs, A->val,
                                                d_status_all.as<int>() + nstat);
        HSS_CHECK_LAUNCH("k_check_finite");
    }
    std::vector<int> status_box;   // box id per flag (-1 - i: top block of instance i)
    Work W(s);
    HSS_CUDA(cudaMemsetAsync(d_tcerr.p, 0, sizeof(int), s));
    Engine eng;
    eng.tc = std::is_same<T, float>::value ? o.tensor_cores : 0;
    eng.bf16 = std::is_same<T, float>::value ? o.sample_bf16 : 0;
    eng.err = d_tcerr.as<int>();
    auto check_tc = [&]() -> int {
        int h = 0;
        HSS_CUDA(cudaMemcpy(&h, d_tcerr.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (h) {
            set_error("hss_factor: a bounded tensor-core wait expired");
            return HSS_ETIMEOUT;
        }
        return HSS_OK;
    };
    F->factor_bytes = 0;
    F->front_flops = 0;
    F->exec_flops = 0;

    auto front_of = [&](int b) {
        FrontDev d{};
        d.foff = foff[b];
        d.ni = t->ni[b];
        d.nb = t->nb[b];
        d.n = d.ni + d.nb;
        d.ioff = t->ioff[b];
        d.iset_off = t->ioff[b];
        d.iperm_off = t->ioff[b];
        d.bset_off = t->boff[b];
        d.leaf = t->child0[b] < 0;
        d.box = b;
        return d;
    };
    // side of each element of a parent front: 0 = in B^child0, 1 = in B^child1
    auto front_dofs = [&](int b, std::vector<int> &dofs, std::vector<int> &sides) {
        dofs.assign(t->iset.begin() + t->ioff[b], t->iset.begin() + t->ioff[b + 1]);
        dofs.insert(dofs.end(), t->bset.begin() + t->boff[b], t->bset.begin() + t->boff[b + 1]);
        sides.assign(dofs.size() / t->bs, 0);
        if (t->child0[b] >= 0) {
            int c0 = t->child0[b];
            std::vector<int> e0;
            for (int i = t->boff[c0]; i < t->boff[c0 + 1]; i += t->bs) e0.push_back(t->bset[i] / t->bs);
            std::sort(e0.begin(), e0.end());
            for (size_t q = 0; q < sides.size(); ++q)
                sides[q] = std::binary_search(e0.begin(), e0.end(), dofs[q * t->bs] / t->bs) ? 0 : 1;
        }
    };

    for (size_t si = 0; si < t->stages.size(); ++si) {
        HSS_HOST("stage");
        const auto &boxes = t->stages[si];
        std::vector<FrontDev> fr;
        std::vector<std::vector<int>> dofs(boxes.size()), sides(boxes.size());
        std::vector<long> poff(boxes.size()), keeph(boxes.size());
        std::vector<int> pn(boxes.size());
        {
            HSS_HOST("stage_fronts");
            for (size_t f = 0; f < boxes.size(); ++f) {
                int b = boxes[f];
                fr.push_back(front_of(b));
                front_dofs(b, dofs[f], sides[f]);
                int par = t->parent[b];
                poff[f] = par >= 0 ? foff[par] : foff_top[t->box_inst[b]];
                pn[f] = par >= 0 ? t->ni[par] + t->nb[par] : ntop_i[t->box_inst[b]];
                keeph[f] = F->keep_h[b];
                const double ni = fr.back().ni, nb = fr.back().nb;
                F->front_flops += 2.0 / 3.0 * ni * ni * ni + 2.0 * ni * ni * nb + 2.0 * nb * nb * ni;
                F->factor_bytes += sizeof(T) * (ni * (ni + nb) + ni * nb);
            }
        }
        W.reset_device();
        ScratchPtr d_fr;
        int *d_status = d_status_all.as<int>() + status_box.size();
        for (int b : boxes) status_box.push_back(b);
        FrontDev *d_frp;
        if ((rc = W.up(fr, &d_frp))) return rc;
        d_fr.p = d_frp;
        {
            HSS_HOST("assemble_stage");
            if ((rc = assemble_stage<T>(A, t, fr, d_fr.as<FrontDev>(), dofs, sides, d_slot.as<int>(), arena, W, s)))
                return rc;
        }
        const bool leaves = std::all_of(boxes.begin(), boxes.end(), [&](int b) { return t->child0[b] < 0; });
        if (structured && !leaves) {
            // Algorithm 1 on every parent front of the stage; a leaf in the same
            // stage eliminates all its pivots in the first phase (n1 = ni)
            std::vector<int> n1(fr.size()), tb(fr.size()), key(fr.size()), nohss(fr.size(), -1);
            std::vector<std::vector<int>> d2(fr.size());
            for (size_t f = 0; f < fr.size(); ++f) {
                const int b = boxes[f], mu = t->child0[b], nu = t->child1[b];
                tb[f] = b;
                key[f] = t->nbox + b;
                if (mu < 0) {
                    n1[f] = t->ni[b];
                    continue;
                }
                int cnt = 0;
                for (int i = t->boff[mu]; i < t->boff[mu + 1]; ++i) cnt += t->fmap[i] < t->ni[b];
                n1[f] = cnt;
                tb[f] = nu;
                key[f] = t->nbox + b;
                d2[f].assign(t->iset.begin() + t->ioff[b] + cnt, t->iset.begin() + t->ioff[b + 1]);
            }
            if ((rc = eliminate_structured<T>(t, o, fr, d_fr.as<FrontDev>(), n1, d2, tb, key, nohss, arena,
                                              d_piv.as<int>(), d_scratch.as<int>(), t->d_iset.as<int>(),
                                              F->d_iperm.as<int>(), d_status, F->exec_flops, F, eng, W, s)))
                return rc;
        } else if ((rc = eliminate_stage<T>(fr, d_fr.as<FrontDev>(), arena, d_piv.as<int>(), d_scratch.as<int>(),
                                            t->d_iset.as<int>(), F->d_iperm.as<int>(), d_status, F->exec_flops, eng,
                                            W, s))) {
            return rc;
        }
        if (o.keep_schur)
            for (size_t f = 0; f < fr.size(); ++f) {
                const FrontDev &d = fr[f];
                if (d.nb == 0) continue;
                HSS_CUDA(cudaMemcpy2DAsync(keep + F->keep_s[d.box], sizeof(T) * d.nb,
                                           arena + d.foff + d.ni + (long)d.n * d.ni, sizeof(T) * d.n,
                                           sizeof(T) * d.nb, d.nb, cudaMemcpyDeviceToDevice, s));
            }
        if ((rc = compress_stage<T>(t, o, fr, boxes, poff, pn, keeph, arena, keep, d_status, (int)fr.size(), F->log,
                                    F, eng, W, s)))
            return rc;
        F->apply.emplace_back();
        build_apply_stage(F->apply.back(), fr, false);
    }
    // ---- top blocks A^(0): cross couplings from A, then full Gauss-Jordan inversion
    {
        HSS_HOST("top");
        std::vector<FrontDev> fr(ninst);
        std::vector<std::vector<int>> dofs(ninst), sides(ninst);
        for (int i = 0; i < ninst; ++i) {
            FrontDev &top = fr[i];
            top = FrontDev{};
            top.foff = foff_top[i];
            top.n = ntop_i[i];
            top.ni = ntop_i[i];
            top.nb = 0;
            top.ioff = ilen + top_off[i];
            top.iset_off = top_off[i];
            top.iperm_off = ilen + top_off[i];
            top.bset_off = 0;
            top.leaf = 0;
            top.box = -1 - i;
            dofs[i].assign(topset.begin() + top_off[i], topset.begin() + top_off[i + 1]);
            sides[i].assign(ntop_i[i] / t->bs, 1);
            for (int q = 0; q < t->nb[t->inst_top[i]] / t->bs; ++q) sides[i][q] = 0;
        }
        W.reset_device();
        ScratchPtr d_fr;
        int *d_status = d_status_all.as<int>() + status_box.size();
        for (int i = 0; i < ninst; ++i) status_box.push_back(-1 - i);
        FrontDev *d_frp;
        if ((rc = W.up(fr, &d_frp))) return rc;
        d_fr.p = d_frp;
        if ((rc = assemble_stage<T>(A, t, fr, d_fr.as<FrontDev>(), dofs, sides, d_slot.as<int>(), arena, W, s)))
            return rc;
        if (structured) {
            // Algorithm 3: S^1 = H^1 eliminated first, S~2 = H^2 - A21 (H^1)^-1 A12
            // compressed over the tree of the second level-1 box
            std::vector<int> n1(ninst), tb(ninst), key(ninst), hb(ninst);
            std::vector<std::vector<int>> d2(ninst);
            for (int i = 0; i < ninst; ++i) {
                n1[i] = t->nb[t->inst_top[i]];
                tb[i] = t->inst_top[i] + 1;
                hb[i] = t->inst_top[i] + 1;
                key[i] = 2 * t->nbox;
            }
            if ((rc = eliminate_structured<T>(t, o, fr, d_fr.as<FrontDev>(), n1, d2, tb, key, hb, arena,
                                              d_piv.as<int>(), d_scratch.as<int>(), F->d_topset.as<int>(),
                                              F->d_iperm.as<int>(), d_status, F->exec_flops, F, eng, W, s)))
                return rc;
        } else if ((rc = eliminate_stage<T>(fr, d_fr.as<FrontDev>(), arena, d_piv.as<int>(), d_scratch.as<int>(),
                                            F->d_topset.as<int>(), F->d_iperm.as<int>(), d_status, F->exec_flops,
                                            eng, W, s))) {
            return rc;
        }
        std::vector<int> hst(nstat + 1);
        if ((rc = factor_readback(hst.data(), d_status_all.p, sizeof(int) * hst.size(), s, F))) return rc;
        if (hst[nstat]) {
            set_error("hss_factor: the matrix A holds a NaN or infinite value");
            return HSS_EINVAL;
        }
        for (size_t q = 0; q < status_box.size(); ++q)
            if (hst[q]) {
                const int b = status_box[q];
                if (b >= 0)
                    set_error("hss_factor: zero pivot in the front of box " + std::to_string(b));
                else
                    set_error(ninst == 1 ? std::string("hss_factor: zero pivot in the top block")
                                         : "hss_factor: zero pivot in the top block of instance " +
                                               std::to_string(-1 - b));
                return HSS_ESINGULAR;
            }
        if (eng.tc && (rc = check_tc())) return rc;
        F->gemm_simt = eng.problems[ENG_SIMT];
        F->gemm_tma = eng.problems[ENG_TMA];
        F->gemm_staged = eng.problems[ENG_STG];
        F->gemm_timed = eng.timed;
        F->gemm_bf16 = eng.problems[ENG_BF16];
        for (int i = 0; i < ninst; ++i) {
            F->front_flops += 2.0 / 3.0 * (double)ntop_i[i] * ntop_i[i] * ntop_i[i];
            F->factor_bytes += sizeof(T) * (double)ntop_i[i] * ntop_i[i];
        }
        F->apply.emplace_back();
        build_apply_stage(F->apply.back(), fr, true);
    }
    // the apply's work items: tuned (packed by the tuner) or the default split
    {
        HSS_HOST("apply_plan");
        if ((rc = o.autotune ? tune_apply(F, s) : pack_apply(F, s))) return rc;
    }
    return factor_readback(nullptr, nullptr, 0, s, F);
}

// ---- one front at a time (test hooks hss_front_eliminate / hss_front_compress):
// the kernels of factor_impl on a front supplied from the host

template <class T>
int front_eliminate_impl(int n, int ni, const double *Fh, int ldf, int tensor_cores, double *out, int ldo,
                         int *perm, cudaStream_t s) {
    Work W(s);
    const size_t nn = (size_t)n * n;
    std::vector<T> host(nn);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) host[i + (size_t)n * j] = (T)Fh[i + (size_t)ldf * j];
    T *arena;
    int *piv, *rperm, *ilist, *iperm, *status, *tcerr;
    std::vector<int> ident(std::max(ni, 1));
    for (int i = 0; i < ni; ++i) ident[i] = i;
    int rc;
    if ((rc = W.up(host, &arena)) || (rc = W.dalloc(std::max(ni, 1), &piv)) ||
        (rc = W.dalloc(std::max(ni, 1), &rperm)) || (rc = W.up(ident, &ilist)) ||
        (rc = W.dalloc(std::max(ni, 1), &iperm)) || (rc = W.dalloc(1, &status)) || (rc = W.dalloc(1, &tcerr)))
        return rc;
    HSS_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    HSS_CUDA(cudaMemsetAsync(tcerr, 0, sizeof(int), s));
    FrontDev d{};
    d.foff = 0;
    d.n = n;
    d.ni = ni;
    d.nb = n - ni;
    d.leaf = 1;
    std::vector<FrontDev> fr{d};
    FrontDev *d_fr;
    if ((rc = W.up(fr, &d_fr))) return rc;
    Engine eng;
    eng.tc = std::is_same<T, float>::value ? tensor_cores : 0;
    eng.err = tcerr;
    double xf = 0;
    if ((rc = eliminate_stage<T>(fr, d_fr, arena, piv, rperm, ilist, iperm, status, xf, eng, W, s))) return rc;
    int hs[2] = {0, 0};
    HSS_CUDA(cudaMemcpyAsync(host.data(), arena, sizeof(T) * nn, cudaMemcpyDeviceToHost, s));
    std::vector<int> hp(std::max(ni, 1));
    HSS_CUDA(cudaMemcpyAsync(hp.data(), iperm, sizeof(int) * hp.size(), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaMemcpyAsync(&hs[0], status, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaMemcpyAsync(&hs[1], tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    if (hs[1]) {
        set_error("hss_front_eliminate: a bounded tensor-core wait expired");
        return HSS_ETIMEOUT;
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) out[i + (size_t)ldo * j] = (double)host[i + (size_t)n * j];
    if (perm)
        for (int i = 0; i < ni; ++i) perm[i] = hp[i];
    if (hs[0]) {
        set_error("hss_front_eliminate: zero pivot");
        return HSS_ESINGULAR;
    }
    return HSS_OK;
}

template <class T>
int front_compress_impl(const hss_tree *t, int box, const double *Sh, int lds, const hss_factor_opts &o, double *Hout,
                        int ldh, int *kmax, int *r, int *rounds, cudaStream_t s) {
    const int nb = t->nb[box];
    const int par = t->parent[box];
    int pn;
    if (par >= 0) {
        pn = t->ni[par] + t->nb[par];
    } else {
        const int b0 = t->inst_top[t->box_inst[box]];
        pn = t->nb[b0] + t->nb[b0 + 1];
    }
    const long sz = ((long)nb * nb + 31) / 32 * 32;
    Work W(s);
    std::vector<T> host((size_t)nb * nb);
    for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) host[i + (size_t)nb * j] = (T)Sh[i + (size_t)lds * j];
    T *arena, *keep;
    int *tcerr;
    int rc;
    if ((rc = W.dalloc(sz + (size_t)pn * pn, &arena)) || (rc = W.dalloc((size_t)nb * nb, &keep)) ||
        (rc = W.dalloc(1, &tcerr)))
        return rc;
    if (nb) HSS_CUDA(cudaMemcpyAsync(arena, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice, s));
    HSS_CUDA(cudaMemsetAsync(tcerr, 0, sizeof(int), s));
    FrontDev d{};
    d.foff = 0;
    d.n = nb;
    d.ni = 0;
    d.nb = nb;
    d.bset_off = t->boff[box];
    d.box = box;
    std::vector<FrontDev> fr{d};
    std::vector<int> boxes{box};
    std::vector<long> poff{sz}, keeph{0};
    std::vector<int> pnv{pn};
    std::vector<FrontLog> logv;
    hss_factor_t tmp;
    Engine eng;
    eng.tc = std::is_same<T, float>::value ? o.tensor_cores : 0;
    eng.bf16 = std::is_same<T, float>::value ? o.sample_bf16 : 0;
    eng.err = tcerr;
    if ((rc = compress_stage<T>(t, o, fr, boxes, poff, pnv, keeph, arena, keep, nullptr, 0, logv, &tmp, eng, W, s)))
        return rc;
    int herr = 0;
    HSS_CUDA(cudaMemcpyAsync(host.data(), keep, sizeof(T) * host.size(), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaMemcpyAsync(&herr, tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("hss_front_compress: a bounded tensor-core wait expired");
        return HSS_ETIMEOUT;
    }
    for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) Hout[i + (size_t)ldh * j] = (double)host[i + (size_t)nb * j];
    const FrontLog &lg = logv.at(0);
    if (kmax) *kmax = lg.kmax;
    if (r) *r = lg.r;
    if (rounds) *rounds = lg.rounds;
    return HSS_OK;
}

}  // namespace
}  // namespace hssnd

using namespace hssnd;

namespace hssnd {
// dst[i] = src[i] + add (row pointers and column indices of one instance moved
// into the block-diagonal union)
__global__ void k_shift_index(const int *__restrict__ src, int n, int add, int *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] + add;
}
}  // namespace hssnd

static int check_factor_opts(const hss_factor_opts &o, const char *who) {
    if (!(o.tol >= 0) || o.r0 < 1 || o.dr < 1 || o.rmax < o.r0 || o.rmax > 128 || o.oversample < 0 ||
        (o.precision != HSS_FP64 && o.precision != HSS_FP32) ||
        (o.cap_policy != HSS_CAP_KEEP && o.cap_policy != HSS_CAP_ACCEPT) || (o.autotune != 0 && o.autotune != 1) ||
        o.probe < 0 || o.probe > PROBE_MAX || (o.probe > 0 && !(o.tol > 0)) || o.tensor_cores < 0 ||
        o.tensor_cores > 3 || (o.sample_bf16 != 0 && o.sample_bf16 != 1) || (o.merge != 0 && o.merge != 1) ||
        (o.merge == 1 && o.probe > 0)) {
        set_error(std::string(who) + ": options out of range (rmax <= 128, tensor_cores 0..3, sample_bf16 0/1, "
                                     "merge 0/1 and no probe with merge = 1)");
        return HSS_EINVAL;
    }
    return HSS_OK;
}

extern "C" int hss_factor_batched(int ninst, const hss_bsr *As, const hss_tree *forest, const hss_factor_opts *opts,
                                  void *stream, hss_factor_t **out) {
    if (!As || !forest || !out || ninst < 1) {
        set_error("hss_factor_batched: null argument or ninst < 1");
        return HSS_EINVAL;
    }
    *out = nullptr;
    hss_factor_opts o;
    hss_factor_opts_default(&o);
    if (opts) o = *opts;
    int rc;
    if ((rc = check_factor_opts(o, "hss_factor_batched"))) return rc;
    if (o.merge != 0) {
        set_error("hss_factor_batched: the structured merge (merge = 1) is for single instances");
        return HSS_EINVAL;
    }
    if (forest->ninst != ninst) {
        set_error("hss_factor_batched: the tree is not a forest of ninst instances (use nd_order_batched)");
        return HSS_EINVAL;
    }
    const int bs = forest->bs;
    for (int i = 0; i < ninst; ++i)
        if (As[i].bs != bs || As[i].nb != forest->inst_elem[i + 1] - forest->inst_elem[i] || !As[i].row_ptr ||
            !As[i].col_idx || !As[i].val) {
            set_error("hss_factor_batched: matrix " + std::to_string(i) + " does not match its tree");
            return HSS_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> nnz(ninst);
    for (int i = 0; i < ninst; ++i)
        HSS_CUDA(cudaMemcpyAsync(&nnz[i], As[i].row_ptr + As[i].nb, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    long nnz_tot = 0;
    for (int v : nnz) nnz_tot += v;
    if (nnz_tot > INT32_MAX) {
        set_error("hss_factor_batched: more than 2^31 blocks in the union");
        return HSS_EINVAL;
    }
    hss_factor_t *F = new hss_factor_t();
    const int nelem = forest->nelem;
    if ((rc = F->b_row.alloc(sizeof(int) * (nelem + 1))) || (rc = F->b_col.alloc(sizeof(int) * std::max(nnz_tot, 1L))) ||
        (rc = F->b_val.alloc(sizeof(double) * std::max(nnz_tot, 1L) * bs * bs))) {
        delete F;
        return rc;
    }
    int *row = F->b_row.as<int>(), *col = F->b_col.as<int>();
    double *val = F->b_val.as<double>();
    long off = 0;
    for (int i = 0; i < ninst; ++i) {
        const int e0 = forest->inst_elem[i];
        if (As[i].nb > 0) {
            HSS_PROF("shift_index", s);
            k_shift_index<<<cdiv(As[i].nb, 256), 256, 0, s>>>(As[i].row_ptr, As[i].nb, (int)off, row + e0);
        }
        if (nnz[i] > 0) {
            {
                HSS_PROF("shift_index", s);
                k_shift_index<<<std::min(cdiv(nnz[i], 256), 1024), 256, 0, s>>>(As[i].col_idx, nnz[i], e0, col + off);
            }
            if (cudaMemcpyAsync(val + off * bs * bs, As[i].val, sizeof(double) * (size_t)nnz[i] * bs * bs,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                delete F;
                return cuda_fail(cudaGetLastError(), "hss_factor_batched: copy of the block values");
            }
        }
        off += nnz[i];
    }
    const int last = (int)nnz_tot;
    if (cudaMemcpyAsync(row + nelem, &last, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        delete F;
        return cuda_fail(cudaGetLastError(), "hss_factor_batched: block-diagonal union");
    }
    F->batched = 1;
    F->bA = hss_bsr{nelem, bs, row, col, val};
    F->tree = forest;
    F->ndof = forest->ndof;
    F->precision = o.precision;
    F->opts = o;
    rc = o.precision == HSS_FP32 ? factor_impl<float>(&F->bA, forest, o, s, F)
                                 : factor_impl<double>(&F->bA, forest, o, s, F);
    if (rc) {
        cudaStreamSynchronize(s);
        delete F;
        return rc;
    }
    *out = F;
    return HSS_OK;
}

extern "C" int hss_factor(const hss_bsr *A, const hss_tree *tree, const hss_factor_opts *opts, void *stream,
                          hss_factor_t **out) {
    if (!A || !tree || !out) {
        set_error("hss_factor: null argument");
        return HSS_EINVAL;
    }
    *out = nullptr;
    hss_factor_opts o;
    hss_factor_opts_default(&o);
    if (opts) o = *opts;
    if (A->nb != tree->nelem || A->bs != tree->bs || !A->val || !(o.tol >= 0) || o.r0 < 1 || o.dr < 1 ||
        o.rmax < o.r0 || o.rmax > 128 || o.oversample < 0 || (o.precision != HSS_FP64 && o.precision != HSS_FP32) ||
        (o.cap_policy != HSS_CAP_KEEP && o.cap_policy != HSS_CAP_ACCEPT) || (o.autotune != 0 && o.autotune != 1) ||
        o.probe < 0 || o.probe > PROBE_MAX || (o.probe > 0 && !(o.tol > 0)) || o.tensor_cores < 0 ||
        o.tensor_cores > 3 || (o.sample_bf16 != 0 && o.sample_bf16 != 1) || (o.merge != 0 && o.merge != 1) ||
        (o.merge == 1 && (o.probe > 0 || tree->ninst != 1))) {
        set_error("hss_factor: invalid argument (matrix/tree mismatch or options out of range; rmax <= 128, "
                  "tensor_cores 0..3, sample_bf16 0/1, merge 0/1; merge = 1 needs probe = 0 and a single "
                  "instance)");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    hss_factor_t *F = new hss_factor_t();
    F->tree = tree;
    F->ndof = tree->ndof;
    F->precision = o.precision;
    F->opts = o;
    const auto t0 = std::chrono::steady_clock::now();
    const double gap0 = prof_readback_gap_ms();
    int rc = o.precision == HSS_FP32 ? factor_impl<float>(A, tree, o, s, F) : factor_impl<double>(A, tree, o, s, F);
    F->host_gap_ms = prof_readback_gap_ms() - gap0;
    F->host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc) {
        cudaStreamSynchronize(s);
        delete F;
        return rc;
    }
    *out = F;
    return HSS_OK;
}

extern "C" int hss_factor_get_info(const hss_factor_t *f, hss_factor_info *info) {
    if (!f || !info) {
        set_error("hss_factor_get_info: null argument");
        return HSS_EINVAL;
    }
    info->factor_bytes = f->factor_bytes;
    info->front_flops = f->front_flops;
    info->executed_flops = f->exec_flops;
    info->max_rank = f->max_rank;
    info->max_r = f->max_r;
    info->rounds = f->rounds;
    info->nfronts = (int)f->log.size();
    info->capped_fronts = f->capped_fronts;
    info->probe_regrown = f->probe_regrown;
    info->gemm_simt = f->gemm_simt;
    info->gemm_tma = f->gemm_tma;
    info->gemm_staged = f->gemm_staged;
    info->gemm_timed = f->gemm_timed;
    info->gemm_bf16 = f->gemm_bf16;
    info->host_syncs = f->host_syncs;
    info->host_sync_ms = f->host_sync_ms;
    info->host_ms = f->host_ms;
    info->host_gap_ms = f->host_gap_ms;
    return HSS_OK;
}

extern "C" int hss_factor_export_log(const hss_factor_t *f, int cap, int *box, int *kmax, int *r, int *rounds) {
    if (!f || cap < 0) {
        set_error("hss_factor_export_log: invalid argument");
        return -1;
    }
    int n = 0;
    for (const auto &lg : f->log) {
        if (lg.nb == 0) continue;
        if (n < cap) {
            if (box) box[n] = lg.box;
            if (kmax) kmax[n] = lg.kmax;
            if (r) r[n] = lg.r;
            if (rounds) rounds[n] = lg.rounds;
        }
        ++n;
    }
    return n;
}

extern "C" int hss_factor_export_front(const hss_factor_t *f, int box, double *S, double *H, int *kmax, int *r) {
    if (!f || box < 0 || box >= f->tree->nbox) {
        set_error("hss_factor_export_front: invalid argument");
        return HSS_EINVAL;
    }
    for (const auto &lg : f->log)
        if (lg.box == box) {
            if (kmax) *kmax = lg.kmax;
            if (r) *r = lg.r;
        }
    if (!S && !H) return HSS_OK;
    if (f->keep_s.empty() || f->keep_s[box] < 0) {
        set_error("hss_factor_export_front: factor built without keep_schur");
        return HSS_EINVAL;
    }
    long nb = f->tree->nb[box];
    size_t cnt = (size_t)nb * nb;
    if (cnt == 0) return HSS_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError(), "export sync");
    for (int which = 0; which < 2; ++which) {
        double *dst = which ? H : S;
        if (!dst) continue;
        long off = which ? f->keep_h[box] : f->keep_s[box];
        if (f->precision == HSS_FP32) {
            std::vector<float> tmp(cnt);
            HSS_CUDA(cudaMemcpy(tmp.data(), f->keep.as<float>() + off, sizeof(float) * cnt, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < cnt; ++i) dst[i] = tmp[i];
        } else {
            HSS_CUDA(cudaMemcpy(dst, f->keep.as<double>() + off, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
        }
    }
    return HSS_OK;
}

extern "C" void hss_factor_destroy(hss_factor_t *f) { delete f; }

extern "C" int hss_front_eliminate(int n, int ni, const double *F, int ldf, int precision, int tensor_cores,
                                   double *out, int ldo, int *perm, void *stream) {
    if (n < 1 || ni < 1 || ni > n || !F || !out || ldf < n || ldo < n ||
        (precision != HSS_FP64 && precision != HSS_FP32) || tensor_cores < 0 || tensor_cores > 3) {
        set_error("hss_front_eliminate: invalid argument");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return precision == HSS_FP32 ? front_eliminate_impl<float>(n, ni, F, ldf, tensor_cores, out, ldo, perm, s)
                                 : front_eliminate_impl<double>(n, ni, F, ldf, 0, out, ldo, perm, s);
}

extern "C" int hss_front_compress(const hss_tree *t, int box, const double *S, int lds, const hss_factor_opts *opts,
                                  double *H, int ldh, int *kmax, int *r, int *rounds, void *stream) {
    hss_factor_opts o;
    hss_factor_opts_default(&o);
    if (opts) o = *opts;
    if (!t || box < 0 || box >= t->nbox || !S || !H || lds < std::max(1, t->nb[box]) ||
        ldh < std::max(1, t->nb[box])) {
        set_error("hss_front_compress: invalid argument");
        return HSS_EINVAL;
    }
    int rc = check_factor_opts(o, "hss_front_compress");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return o.precision == HSS_FP32 ? front_compress_impl<float>(t, box, S, lds, o, H, ldh, kmax, r, rounds, s)
                                   : front_compress_impl<double>(t, box, S, lds, o, H, ldh, kmax, r, rounds, s);
}

extern "C" int hss_gemm_tuner_read(int idx, long long *key, int *engine, float *ms_simt, float *ms_tc) {
    std::lock_guard<std::mutex> lk(g_eng_mu);
    if (idx < 0) return (int)g_eng_order.size();
    if (idx >= (int)g_eng_order.size()) {
        set_error("hss_gemm_tuner_read: index out of range");
        return -HSS_EINVAL;
    }
    const uint64_t k = g_eng_order[idx];
    const EngChoice &c = g_eng_choice[k];
    if (key) *key = (long long)k;
    if (engine) *engine = c.engine;
    if (ms_simt) *ms_simt = c.ms_simt;
    if (ms_tc) *ms_tc = c.ms_tc;
    return HSS_OK;
}
