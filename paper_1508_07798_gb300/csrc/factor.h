// The factorization handle.
#pragma once
#include <memory>

#include "front.h"
#include "internal.h"

namespace hssnd {

constexpr int APPLY_ROWS = 32;

constexpr int APPLY_CHUNK = 64;   // columns per warp work item of the apply
constexpr int APPLY_SUB_MIN = 256;   // fronts of the level that roots the apply's subtrees (one CTA each)
constexpr int APPLY_SUB_MAXN = 192;  // largest front (n) of the levels the subtree launch takes

struct ApplyItem {
    int front;        // stage-local front index
    int row0;         // first of the 32 rows
    int c0, c1;       // column range of this item
    int tile;         // row-tile index inside the stage (ticket slot)
    int first;        // item index of the tile's first chunk
    int nchunk;       // chunks of this tile
};

// Per level (and the top block): fronts and the row tiles of the apply.
struct ApplyStage {
    bool top = false;
    int nfronts = 0;
    std::vector<FrontDev> h_fronts;       // host copies, packed into the factor's apply buffer
    int chunk[2] = {APPLY_CHUNK, APPLY_CHUNK};   // columns per work item of the forward / backward sweep
    FrontDev *d_fronts = nullptr;
    ApplyItem *d_fwd = nullptr, *d_bwd = nullptr;
    int nfwd = 0, nbwd = 0;               // work items (warps) of the two sweeps
    long part_fwd = 0, part_bwd = 0;      // offsets (in items) into the partial-sum buffer
    int tk_fwd = 0, tk_bwd = 0;           // offsets into the ticket array
    double fwd_bytes = 0, bwd_bytes = 0;  // factor entries read (x8 bytes in FP64)
    double fwd_vec = 0, bwd_vec = 0;      // vector entries read + written per right-hand side
};

// Vector arguments of one apply, read by the sweep kernels from device memory
// (so that one captured graph serves every call).
struct ApplyParams {
    const double *x;
    long ldx;
    double *w;
    long ldw;
    double *tv;
    long ldt;
    int nrhs;
};

constexpr int APPLY_RB = 8;   // right-hand sides per sweep of the multi-RHS apply (factor read once per 8)

struct FrontLog {   // per-front record (rank logging, Sec. 5 empirical cost)
    int box, level, ni, nb, r, rounds, kmax, nnodes;
};

int apply_factor(const hss_factor_t *f, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s);
// Work items of every apply stage from its fronts and column chunks, packed
// into one device buffer with the partial-sum and ticket arrays (drops any
// captured graph).
int pack_apply(hss_factor_t *F, cudaStream_t s);
// Chooses each stage's forward and backward column chunk by timing the
// candidates (process-wide cache keyed by the stage's front shapes).
int tune_apply(hss_factor_t *F, cudaStream_t s);
int ilu_apply(const hss_ilu_t *M, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s);
long ilu_ndof(const hss_ilu_t *M);
int spmv(const hss_bsr *A, int nrhs, const double *x, long ldx, double *y, long ldy, cudaStream_t s);

// Right preconditioner of the Krylov solvers: the HSS factorization, block
// ILU(0), or none (both null).
struct Precond {
    const hss_factor_t *hss = nullptr;
    const hss_ilu_t *ilu = nullptr;
    bool none() const { return !hss && !ilu; }
};
inline int precond_apply(const Precond &P, int nrhs, const double *x, long ldx, double *y, long ldy,
                         cudaStream_t s) {
    return P.hss ? apply_factor(P.hss, nrhs, x, ldx, y, ldy, s) : ilu_apply(P.ilu, nrhs, x, ldx, y, ldy, s);
}

int fgmres_lockstep(const hss_bsr *A, const Precond &pc, const std::vector<int> &inst_dof, int nrhs,
                    const double *b, int ldb, double *x, int ldx, const fgmres_opts &o, fgmres_stats *stats,
                    std::vector<std::vector<double>> *hist, cudaStream_t s);

}  // namespace hssnd

struct hss_factor_t {
    const hss_tree *tree = nullptr;
    int ndof = 0;
    int precision = HSS_FP64;
    hss_factor_opts opts{};
    hssnd::DevBuf arena;         // all fronts and the top block (T = double or float)
    hssnd::DevBuf d_iperm;       // gather lists of the apply (iset_len + ntop)
    hssnd::DevBuf d_topset;      // [B^1 ; B^2]
    hssnd::DevBuf tvec;          // apply scratch (N x nrhs)
    hssnd::DevBuf keep;          // optional copies of S and H per front
    std::vector<long> keep_s, keep_h;  // per box offsets (-1: none)
    std::vector<hssnd::ApplyStage> apply;
    std::vector<hssnd::FrontLog> log;
    int ntop = 0;
    double factor_bytes = 0, front_flops = 0, exec_flops = 0;
    int max_rank = 0, max_r = 0, rounds = 0;
    int capped_fronts = 0;   // fronts that kept S because the sample width reached rmax
    int probe_regrown = 0;   // sampling rounds added by failed residual probes
    long gemm_simt = 0, gemm_tma = 0, gemm_staged = 0, gemm_timed = 0;   // GEMM problems per engine, tuner timings
    long gemm_bf16 = 0;      // sampling products on the BF16 tensor-core kernel
    long host_syncs = 0;       // blocking read-backs of the factorization
    double host_sync_ms = 0;   // host time spent waiting in them
    double host_ms = 0;        // host time of the whole call
    double host_gap_ms = 0;    // host time from each read-back to the next kernel launch (device idle)
    // captured apply sweeps (slot 0: one right-hand side, slot 1: blocks of APPLY_RB)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_kernels[2] = {0, 0};
    hssnd::DevBuf d_aparams;
    hssnd::DevBuf d_apart;       // partial sums of split apply tiles (items x 32 x 4)
    hssnd::DevBuf d_tickets;     // one ticket counter per split tile
    hssnd::DevBuf apply_buf;     // fronts and work items of every apply stage, one allocation
    // subtree part of the apply: stages [0, sub_nst) (the deepest levels) run
    // as one launch per direction, one CTA per subtree rooted in stage
    // sub_nst - 1; items and per-(subtree, stage) offsets live in apply_buf
    int sub_nst = 0, sub_n = 0;
    hssnd::FrontDev *d_sub_fronts = nullptr;
    hssnd::ApplyItem *d_sub_fwd = nullptr, *d_sub_bwd = nullptr;
    int *d_sub_off_fwd = nullptr, *d_sub_off_bwd = nullptr;
    // batched factor (hss_factor_batched): device copy of the block-diagonal
    // union of the instances' matrices, used by the batched solver
    int batched = 0;
    hss_bsr bA{};
    hssnd::DevBuf b_row, b_col, b_val;
    template <class T> T *arena_ptr() const { return arena.as<T>(); }
    // algorithmic bytes of one apply: factor entries once, vector traffic per right-hand side
    double apply_bytes(int nrhs) const {
        double b = 0;
        for (const auto &st : apply)
            b += (st.fwd_bytes + st.bwd_bytes) * (precision == HSS_FP32 ? 0.5 : 1.0) +
                 (st.fwd_vec + st.bwd_vec) * 8.0 * nrhs;
        return b + 2.0 * 8.0 * ndof * nrhs;   // copy-in
    }
    ~hss_factor_t() {
        for (auto &g : gexec)
            if (g) cudaGraphExecDestroy(g);
    }
};
