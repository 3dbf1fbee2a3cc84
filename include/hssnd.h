/*
 * hssnd.h -- C ABI of libhssnd.so, a GB300 (sm_103a) implementation of the
 * preconditioner of Gatto & Hesthaven, "A Preconditioner Based on Low-Rank
 * Approximation of Schur Complements" (arXiv 1508.07798):
 *
 *   nd_order      nested-dissection box tree and interior/boundary dof sets
 *                 (paper Sec. 4.0, graph (1), eq. (30)/(31) ordering)
 *   hss_factor    approximate LDM^t factorization, Algorithm 2: fronts are
 *                 eliminated level by level (eq. (32)), each Schur complement is
 *                 replaced by a randomized HSS/ID approximant (Theorem 1), the top
 *                 block A^(0) of eq. (36) is inverted
 *   hss_apply     y = M^-t D^-1 L^-1 x (end of Sec. 4.2)
 *   fgmres_solve  right-preconditioned restarted flexible GMRES (Sec. 5 measures
 *                 the preconditioner in GMRES iterations)
 *
 * Conventions for every call:
 *   - Pointers named d_* or documented as "device" are CUDA device pointers;
 *     everything else is host memory.  The caller owns all buffers it passes;
 *     the library owns the opaque handles (hss_tree, hss_factor_t) and the
 *     device memory behind them until the matching *_destroy call.
 *   - No call modifies the matrix A.
 *   - Dense vectors/matrices are column-major with a leading dimension (ld >= N).
 *     Vectors use the ORIGINAL dof numbering (global dof = element*bs + local).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is stream-ordered; calls that must size allocations or report
 *     statistics synchronize the stream (stated per call).
 *   - Every int-returning call returns HSS_OK (0) or an error code; no
 *     exception crosses the ABI.  hss_last_error() describes the last error of
 *     the calling thread.  Handles are not thread-safe.
 *   - The library never falls back to a CPU implementation: without a usable
 *     CUDA device every compute call fails with HSS_ECUDA.
 */
#ifndef HSSND_H
#define HSSND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HSS_OK = 0,
    HSS_EINVAL = 1,      /* invalid argument (sizes, null pointers, NaN/Inf in A) */
    HSS_ENOMEM = 2,      /* device allocation failed or over the memory budget   */
    HSS_ESINGULAR = 3,   /* zero pivot in a front; the box id is in hss_last_error */
    HSS_ENOCONV = 4,     /* FGMRES hit maxit; x holds the last iterate            */
    HSS_ETIMEOUT = 5,    /* a bounded device-side wait expired                    */
    HSS_ECUDA = 6        /* CUDA runtime error (including: no device)            */
};

enum { HSS_SCHEME_BOX = 0, HSS_SCHEME_HSLAB = 1, HSS_SCHEME_VSLAB = 2 };
enum { HSS_FP64 = 0, HSS_FP32 = 1 };

/* Square block-sparse matrix, DEVICE pointers.  nb block rows (one per
 * element), bs x bs dense blocks stored row-major (row = test function),
 * block columns sorted ascending in each block row. */
typedef struct hss_bsr {
    int nb;
    int bs;
    const int *row_ptr;     /* [nb+1] */
    const int *col_idx;     /* [nnzb] */
    const double *val;      /* [nnzb*bs*bs] */
} hss_bsr;

/* Structured element grid on the unit square/cube: element
 * e = ix + n[0]*(iy + n[1]*iz), bs = (p+1)^dim dofs per element. */
typedef struct hss_mesh {
    int dim;
    int n[3];
    int p;
} hss_mesh;

typedef struct hss_nd_opts {
    int leaf_max;           /* a box with <= leaf_max dofs (or one element) is a leaf; default 64 */
    int scheme;             /* HSS_SCHEME_*; default BOX */
} hss_nd_opts;

typedef struct hss_factor_opts {
    double tol;             /* relative ID tolerance per interpolative decomposition; default 1e-6 */
    int compress;           /* 1: replace each Schur complement by its HSS approximant (default);
                               0: exact LDM^t (no approximation) */
    int r0;                 /* initial sample width; default 32 */
    int dr;                 /* sample width growth step; default 32 */
    int rmax;               /* largest sample width; default 96 */
    int oversample;         /* p of Theorem 1; a node rank above r - p triggers growth; default 10 */
    int precision;          /* HSS_FP64 (default) or HSS_FP32 (mixed form) */
    uint64_t seed;          /* seed of the +-1 test matrices; default 0 */
    int keep_schur;         /* 1: keep a copy of every front's S and H for hss_factor_export_front */
    int tensor_cores;       /* FP32 form only: 0 (default) SIMT FMA; 1 tcgen05 TF32 with the three-product
                               hi/lo split (FP32 accuracy) for products with M, K >= 128 and N >= 32 (the
                               sampling products and the K = 256 updates of the blocked sweep), operands
                               brought in by TMA where they are 16-byte aligned with leading dimensions
                               that are multiples of 4 (front sizes divisible by 4), staged by the threads
                               otherwise; 2 tcgen05 with a single TF32 product (threads staging); 3 per
                               shape class (operand forms, m, n, k rounded up to powers of two) of the
                               problems the TMA-fed kernel can take: SIMT or that kernel, timed on a scratch
                               C the first time the class appears (the tensor cores need a 15% lead) and
                               cached for the process; other problems on SIMT */
    const int *r_init;      /* HOST array of one initial sample width per box (NULL, the default: r0 for
                               every front), e.g. from hss_rank_model_predict; the adaptive growth by dr
                               still applies whenever a rank exceeds r - oversample */
    int cap_policy;         /* a front whose rank still exceeds r - oversample when r + dr > rmax stops the
                               growth: HSS_CAP_KEEP (default) keeps S itself (Theorem 1's bound needs k + p
                               samples); HSS_CAP_ACCEPT keeps the approximant built from the r samples it
                               has (ranks up to r, no error bound) -- with r0 = rmax = l this is the fixed
                               anticipated rank l of the experiments of Sec. 5 */
    int autotune;           /* 1: choose each level's apply work split (columns per work item of the
                               forward and backward sweeps, from 32, 64, 128, 256) by timing the candidates
                               on the factor's stream; choices are cached for the process, keyed by the
                               level's front shapes, so a structure is timed once.  0 (default): 64.  The
                               split changes only the summation order of the apply. */
    int probe;              /* residual probe of every approximant the rank test accepts (the fallback check
                               of learned widths): with W = `probe` +-1 vectors (0 = off, the default; at
                               most 8) from stream 2 of the counter generator, a front with
                               ||(S - H) W||_F > 10 tol depth ||S W||_F (depth = depth of its HSS tree, at
                               least 1) samples again with r + dr while r + dr <= rmax.  Needs tol > 0. */
    int sample_bf16;        /* FP32 form: 1 runs the sampling products Y = S Omega, Z = S^t Psi of every front
                               whose S the TMA can address (front sizes divisible by 4, |B| >= 128) on
                               tcgen05 kind::f16 with FP32 accumulation: S is split into three BF16 terms
                               (x ~ t0 + t1 + t2, each the BF16 rounding of what the previous left, about
                               FP32 accuracy) and the +-1 test matrix is exact in BF16.  0 (default): the
                               sampling follows tensor_cores. */
    int merge;              /* 0 (default): the interior block of every front factored densely (reading R1).
                               1: the structured merge of Algorithm 1 (eq. (37)) and Algorithm 3: in a parent
                               front the first child's interior pivots are eliminated first, the second
                               Schur complement S~ = S2 - A21 S1^-1 A12 left in the trailing interior block
                               is replaced by its HSS approximant (Theorem 1, tree: the second child's
                               subtree restricted to those dofs, test-matrix key nbox + box; for the top
                               block the second level-1 box's tree, key 2 nbox), then the rest; the front is
                               thus factored with A_ii + blockdiag(0, H~ - S~) in place of A_ii, whose inverse
                               is eq. (37)'s block solve.  Dense fronts throughout (the approximation of R2,
                               not its complexity).  Needs probe = 0 and a single instance. */
} hss_factor_opts;

enum { HSS_CAP_KEEP = 0, HSS_CAP_ACCEPT = 1 };

typedef struct fgmres_opts {
    int restart;            /* default 30 */
    double rtol;            /* relative residual target ||b - A x|| / ||b||; default 1e-8 */
    int maxit;              /* total Arnoldi steps per right-hand side; default 1000 */
} fgmres_opts;

typedef struct fgmres_stats {
    int iters;              /* Arnoldi steps, summed over right-hand sides */
    int max_iters;          /* largest per right-hand side */
    double relres;          /* largest final true relative residual over right-hand sides */
    int converged;          /* 1 when every right-hand side reached rtol */
} fgmres_stats;

typedef struct hss_tree hss_tree;
typedef struct hss_factor_t hss_factor_t;
typedef struct hss_ilu_t hss_ilu_t;

/* Default option values (host structs). */
void hss_nd_opts_default(hss_nd_opts *o);
void hss_factor_opts_default(hss_factor_opts *o);
void fgmres_opts_default(fgmres_opts *o);

/* Sec. 4.0: build the box tree of `mesh` (recursive bisection of the element
 * grid; at a tie the last axis is cut; the lower child gets floor(n/2)
 * elements), classify each box's dofs as boundary (coupled by a stored block of
 * A to a dof outside the box) or interior, and form the eq. (31) elimination
 * order.  `A` (device) supplies the coupling structure only.  The element
 * flags and set compaction run on the device; the call synchronizes `stream`
 * once to size the sets.  *out receives a new handle.  Errors: HSS_EINVAL
 * (mesh/BSR mismatch, fewer than two elements), HSS_ENOMEM, HSS_ECUDA. */
int nd_order(const hss_mesh *mesh, const hss_bsr *A, const hss_nd_opts *opts,
             void *stream, hss_tree **out);

/* Sizes of a tree: N, number of boxes, deepest level, total lengths of the
 * concatenated interior / boundary set arrays. */
typedef struct hss_tree_desc {
    int ndof, nbox, maxlev, iset_len, bset_len, bs;
} hss_tree_desc;
int hss_tree_info(const hss_tree *t, hss_tree_desc *d);

/* Copy the tree to HOST arrays (any pointer may be NULL to skip it).
 * Per box (length nbox): level, parent (-1 for level 1), child0/child1 (-1 at
 * leaves), ni, nb (sizes of the I and B sets), ioff, boff (offsets of the sets
 * inside iset/bset), lohi (6 ints per box: lo[3], hi[3] element ranges).
 * iset[iset_len], bset[bset_len]: global dof ids, boxes concatenated in id order;
 * fmap[bset_len]: position of each B dof inside its parent front [I^;B^] (level 1:
 * inside the top block [B^1;B^2]); perm[ndof]: eq. (31) elimination order. */
int hss_tree_export(const hss_tree *t, int *level, int *parent, int *child0, int *child1,
                    int *ni, int *nb, int *ioff, int *boff, int *lohi,
                    int *iset, int *bset, int *fmap, int *perm);

/* Algorithm 2: eliminate every front level by level (leaves first), compress
 * each Schur complement S = F_bb - F_bi F_ii^-1 F_ib (eq. (32)) to its
 * randomized HSS approximant H (Theorem 1; ID with relative tolerance
 * opts->tol, +-1 test matrices from a counter hash), assemble the parent front
 * from H^mu, H^nu and A(B^mu, B^nu), and invert the top block
 * A^(0) = [[H^1, A12], [A21, H^2]] (eq. (36)).  The factor keeps, per front,
 * F_ii^-1, -F_bi F_ii^-1 and F_ii^-1 F_ib in FP64 (or FP32 with
 * precision = HSS_FP32).  Synchronizes `stream` once per tree level (rank
 * decisions).  Errors: HSS_EINVAL (also when a stored value of A is NaN or
 * infinite: a device scan of A's values, reported at the end of the call),
 * HSS_ENOMEM, HSS_ESINGULAR (box id in hss_last_error), HSS_ECUDA. */
int hss_factor(const hss_bsr *A, const hss_tree *tree, const hss_factor_opts *opts,
               void *stream, hss_factor_t **out);

/* Statistics of a factorization (host): stored factor bytes, algorithmic
 * flops of the front eliminations (2/3 ni^3 + 2 ni^2 nb + 2 nb^2 ni summed),
 * sample rounds, largest HSS rank and sample width, and the number of fronts
 * that kept their Schur complement S uncompressed because the sample width
 * reached opts.rmax while some rank still exceeded r - oversample (Theorem 1
 * needs k + p samples for its error bound). */
typedef struct hss_factor_info {
    double factor_bytes;
    double front_flops;
    double executed_flops;
    int max_rank;
    int max_r;
    int rounds;
    int nfronts;
    int capped_fronts;
    int probe_regrown;      /* sampling rounds added because a residual probe failed */
    long gemm_simt;         /* GEMM problems (one per front and update/sampling step) run on SIMT FMA */
    long gemm_tma;          /* ... on tcgen05 with TMA-fed operands */
    long gemm_staged;       /* ... on tcgen05 with thread-staged operands */
    long gemm_timed;        /* problems the GEMM engine tuner timed (tensor_cores = 3) */
    long gemm_bf16;         /* sampling products run on the BF16 tensor-core kernel (sample_bf16) */
    long host_syncs;        /* blocking device->host read-backs inside the call (ranks of each
                               sampling round, probe norms, pivot flags, the end of the call) */
    double host_sync_ms;    /* host time spent waiting in them */
    double host_ms;         /* host time of the whole call; host_ms - host_sync_ms is the host's
                               own work (planning, launches), during which the device may idle */
    double host_gap_ms;     /* host time from each read-back to the next kernel launch: the
                               device has no work queued meanwhile (the last read-back of the
                               call, with nothing after it, counts toward the next call) */
} hss_factor_info;
int hss_factor_get_info(const hss_factor_t *f, hss_factor_info *info);

/* Test/inspection hook (needs opts.keep_schur = 1): copy box `box`'s Schur
 * complement S (nb x nb, column-major, before compression) and its
 * approximant H to HOST buffers (either may be NULL), plus the largest rank
 * and final sample width of that front.  Synchronizes the stream. */
int hss_factor_export_front(const hss_factor_t *f, int box, double *S, double *H,
                            int *kmax, int *r);

/* y = M^-t D^-1 L^-1 x for nrhs columns (x, y DEVICE, column-major, leading
 * dimensions ldx, ldy >= N, original dof order; x and y may alias).  Forward
 * sweep over the levels, top block, backward sweep.  Asynchronous on `stream`.
 * Errors: HSS_EINVAL, HSS_ENOMEM (workspace for a larger nrhs), HSS_ECUDA. */
int hss_apply(const hss_factor_t *f, int nrhs, const double *x, int ldx, double *y, int ldy,
              void *stream);

/* Test hooks: one step of Algorithm 2 on one front supplied from the host,
 * through the same kernels hss_factor runs, so each step can be checked on
 * its own against a reference that starts from the same input.
 *
 * hss_front_eliminate: the elimination of eq. (32) on the dense front
 * F = [F_ii F_ib; F_bi F_bb] (HOST, n x n column-major, ld ldf >= n; the
 * first ni rows/columns are I, 1 <= ni <= n): the Gauss-Jordan sweep with
 * partial row pivoting inside I that hss_factor uses (fronts with n >= 2048
 * take its blocked form).  out (HOST, n x n, ld ldo >= n) receives the
 * transformed front [F_ii^-1 P^t, W; -F_bi F_ii^-1 P^t, S] with
 * W = F_ii^-1 F_ib and S = F_bb - F_bi W; perm (HOST, ni ints, may be NULL)
 * gives P: column j of the first ni columns belongs to I row perm[j].
 * precision HSS_FP64 or HSS_FP32 (tensor_cores 0..3 as in hss_factor_opts,
 * FP32 only).  Synchronizes `stream`.  Errors: HSS_EINVAL, HSS_ESINGULAR (zero
 * pivot; out is still written), HSS_ENOMEM, HSS_ETIMEOUT, HSS_ECUDA.
 *
 * hss_front_compress: Theorem 1's randomized HSS construction of the Schur
 * complement S (HOST, nb x nb column-major, ld lds >= nb, nb = |B| of `box`
 * in tree t) exactly as hss_factor compresses box `box`: its HSS tree, its
 * test-matrix counters (opts->seed, the box id), the width schedule, cap
 * policy and residual probe of *opts (NULL: defaults; r_init, when given, is
 * read at index `box`).  H (HOST, nb x nb, ld ldh >= nb) receives the
 * approximant (S itself for a single-node HSS tree or compress = 0); kmax,
 * r, rounds (HOST, may be NULL): largest node rank, final sample width,
 * sampling rounds (0 when not compressed).  Synchronizes `stream`.
 * Errors: HSS_EINVAL, HSS_ENOMEM, HSS_ETIMEOUT, HSS_ECUDA. */
int hss_front_eliminate(int n, int ni, const double *F, int ldf, int precision, int tensor_cores, double *out,
                        int ldo, int *perm, void *stream);
int hss_front_compress(const hss_tree *t, int box, const double *S, int lds, const hss_factor_opts *opts,
                       double *H, int ldh, int *kmax, int *r, int *rounds, void *stream);

/* C = alpha A B + beta C in FP32, DEVICE column-major m x k, k x n, m x n
 * (the GEMM of the FP32 form, exposed for testing and reuse).  engine: 0 SIMT
 * FMA; 1 tcgen05 TF32 with the three-product hi/lo split, operands staged by
 * the threads; 2 tcgen05 single TF32; 3 tcgen05 TF32 with the hi/lo split,
 * operands brought in by TMA (cp.async.bulk.tensor) through a 3-stage ring
 * (needs A and B 16-byte aligned and lda, ldb multiples of 4; other operands
 * run on engine 1).  No counterpart in the paper (a building block of eq. (32)'s update).
 * k = 0 gives C = beta C with every engine.  Synchronizes `stream`;
 * HSS_ETIMEOUT if a bounded tensor-core wait expired. */
int hss_gemm_f32(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                 float alpha, float beta, int engine, void *stream);

/* hss_gemm_f32 without any memory allocation.  No counterpart in the paper.
 * Same arguments, layout, engines 0-2 and result as hss_gemm_f32 (engine 3,
 * whose tensor maps are built per call, is not offered here); the difference
 * is where the launch records live: hss_gemm_f32 puts its GEMM descriptor,
 * tile list and tensor-core timeout flag in workspace it allocates per call,
 * this variant keeps them in one fixed device array inside the library
 * (256-byte aligned, 512 + 12 * HSS_GEMM_STATIC_MAX_TILES bytes, about
 * 193 KB), so it calls no allocator of any kind (no cudaMalloc/cudaFree, no
 * pinned host buffer, no allocating library routine).  It is for callers
 * that may not allocate: code that runs while a memory pool or allocator is
 * being trimmed or rebuilt (an allocation there re-enters it), code with a
 * fixed device-memory budget that must leave the heap untouched, and code
 * that must not block the device, which freeing workspace does.
 * Limit: the product is cut into tiles (64 x 64 for engine 0, 128 x 128 for
 * engines 1 and 2) and at most HSS_GEMM_STATIC_MAX_TILES tiles fit, e.g.
 * m = n = 8192 with engine 0, 16384 with engines 1 and 2; a larger m x n
 * returns HSS_EINVAL with the tile count in hss_last_error().
 * k = 0 gives C = beta C with every engine and uses no tile records (no
 * tile limit).
 * Nothing in the scratch has to start at zero: each call writes the
 * descriptor, tile list and a cleared timeout flag on `stream` before the
 * GEMM reads them.  There is one array per device: two calls that overlap in
 * time (on different streams or host threads) race on it and give undefined
 * results; callers serialize them.  The first call on a device, whatever its
 * engine, does all one-time setup of that device: it looks up the array's
 * device address (cudaGetSymbolAddress), loads every kernel this call can
 * launch and sets the tensor-core kernel's shared-memory attribute.  A caller
 * that wants that setup out of a timed or restricted region makes one small
 * call first.  The optional event timing of hss_profile_enable creates CUDA
 * events: leave it off where nothing may be allocated.
 * Synchronizes `stream`; HSS_ETIMEOUT if a bounded tensor-core wait expired,
 * HSS_ECUDA if the address lookup or a launch failed. */
#define HSS_GEMM_STATIC_MAX_TILES 16384
int hss_gemm_f32_static(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C,
                        int ldc, float alpha, float beta, int engine, void *stream);

/* y = A x for nrhs columns (DEVICE, column-major).  Asynchronous. */
int hss_spmv(const hss_bsr *A, int nrhs, const double *x, int ldx, double *y, int ldy,
             void *stream);

/* Right-preconditioned flexible GMRES(restart) for A x = b, one Krylov space
 * per right-hand side.  f == NULL means no preconditioner.  b, x DEVICE
 * (column-major; x holds x0 on entry and the iterate on exit).  FP64 Arnoldi
 * with classical Gram-Schmidt applied twice, Givens rotations on the device;
 * stops when the true FP64 residual, recomputed at every restart, is
 * <= rtol ||b||.  With several right-hand sides their Krylov processes
 * advance in lock step (one multi-vector apply and SpMV per Arnoldi step;
 * a process that has stopped is masked).  Synchronizes once per Arnoldi step
 * and fills *stats (HOST, may be NULL).  Returns HSS_ENOCONV when some
 * right-hand side did not reach rtol within maxit steps. */
int fgmres_solve(const hss_bsr *A, const hss_factor_t *f, int nrhs, const double *b, int ldb,
                 double *x, int ldx, const fgmres_opts *opts, fgmres_stats *stats, void *stream);

/* ---- Batched form: many independent problems in one pass over the levels.
 * The paper treats one problem; Algorithm 2 runs unchanged per instance and
 * only the scheduling is shared.  All instances must have the same block size
 * bs (group instances by dim and p).
 *
 * nd_order_batched: orders every instance as nd_order does and returns one
 * forest: the instances' boxes, elements and dofs are concatenated in instance
 * order (instance i's dof d is forest dof D_i + d, D_i the sum of the earlier
 * instances' dof counts), and tree level l holds level l of every instance.
 * meshes and As are HOST arrays of ninst entries (As' pointers are device
 * pointers).  Synchronizes `stream`.  Errors: as nd_order (the failing
 * instance is named in hss_last_error), HSS_EINVAL when block sizes differ. */
int nd_order_batched(int ninst, const hss_mesh *meshes, const hss_bsr *As, const hss_nd_opts *opts,
                     void *stream, hss_tree **out);

/* hss_factor_batched: Algorithm 2 on every instance of a forest, one tree
 * level of all instances at a time (each elimination, sampling, ID and
 * expansion launch covers the fronts of every instance at that level).  Each
 * instance keeps its own top block A^(0) (eq. (36)) and its test matrices are
 * counted by the instance's own box ids, so instance i's part of the factor
 * is the one hss_factor computes for instance i alone.  The factor keeps a
 * device copy of the block-diagonal union of As (HOST array of ninst
 * matrices).  hss_apply on the result applies every instance's
 * preconditioner to a forest vector; hss_factor_export_front takes forest box
 * ids.  Synchronizes `stream`.  Errors: as hss_factor. */
int hss_factor_batched(int ninst, const hss_bsr *As, const hss_tree *forest, const hss_factor_opts *opts,
                       void *stream, hss_factor_t **out);

/* fgmres_solve_batched: the FGMRES(restart) of fgmres_solve for every
 * (instance, right-hand side) pair of a batched factor, each an independent
 * Krylov process with its own Hessenberg matrix, rotations, stopping test and
 * restarts, all advanced in lock step so that an Arnoldi step costs one
 * hss_apply and one SpMV over the whole batch (processes that have stopped
 * are masked).  b, x: DEVICE forest vectors, ndof x nrhs column-major
 * (ldb, ldx >= ndof); x holds x0 on entry and the solutions on return.
 * stats: HOST array of ninst entries (per instance, over its right-hand
 * sides), may be NULL.  Synchronizes `stream` once per Arnoldi step.
 * Returns HSS_ENOCONV when a process reached maxit first. */
int fgmres_solve_batched(const hss_factor_t *f, int nrhs, const double *b, int ldb, double *x, int ldx,
                         const fgmres_opts *opts, fgmres_stats *stats, void *stream);

/* ---- Learned sample widths (no counterpart in the paper: Theorem 1 needs
 * k + p samples and the paper grows the width until the ranks fit).  A small
 * MLP predicts each front's largest HSS rank k before sampling, so the first
 * sampling round usually suffices; the adaptive growth remains the fallback
 * whenever a rank exceeds r - oversample (the oversampling margin that
 * Theorem 1's bound needs).
 *
 * Features per box (hss_rank_features, HOST out, nbox x 6 row-major):
 * log(1 + |B|), tree level, kappa * h, p, mean and variance of c over the
 * box's elements (c_elem: HOST array per element, NULL meaning c = 1).
 * Network: standardised features -> three ReLU layers of 64 -> one output,
 * the standardised log(1 + k).  Parameters (HSS_RANK_NPARAMS floats, layout
 * W1 (64 x 6, row per unit), b1, W2 (64 x 64), b2, W3 (64 x 64), b3, W4 (64),
 * b4) and the standardisation (14 floats: feature means[6], standard
 * deviations[6], target mean, target standard deviation). */
#define HSS_RANK_FEATURES 6
#define HSS_RANK_HIDDEN 64
#define HSS_RANK_NPARAMS 8833
typedef struct hss_rank_model hss_rank_model;
int hss_rank_features(const hss_tree *t, const double *c_elem, double kappa_h, float *feat);
/* New model: weights uniform in +-sqrt(6 / fan_in) from the counter hash of
 * `seed`, biases 0, identity standardisation. */
int hss_rank_model_create(uint64_t seed, hss_rank_model **out);
void hss_rank_model_destroy(hss_rank_model *m);
/* Copy the parameters / standardisation out (HOST; either may be NULL) or in
 * (setting parameters also clears the Adam state). */
int hss_rank_model_get(const hss_rank_model *m, float *params, float *norm);
int hss_rank_model_set(hss_rank_model *m, const float *params, const float *norm);
/* Standardisation from n training samples: feat DEVICE n x 6 row-major,
 * target DEVICE n values of log(1 + k).  Means and population standard
 * deviations (1 where zero).  Synchronizes `stream`. */
int hss_rank_model_fit_norm(hss_rank_model *m, int n, const float *feat, const float *target, void *stream);
/* Mean squared error over n samples and its gradient (HOST, NPARAMS floats;
 * either may be NULL) at the current parameters.  Synchronizes `stream`. */
int hss_rank_model_loss_grad(hss_rank_model *m, int n, const float *feat, const float *target, float *loss,
                             float *grad, void *stream);
/* Adam (lr, 0.9, 0.999, 1e-8) for `epochs` passes over the data in minibatches
 * of `batch` samples, order per epoch from the counter hash of `seed`; the
 * final mean squared error over all samples goes to *final_loss (may be NULL).
 * FP32 forward and backward kernels on the device. */
int hss_rank_model_train(hss_rank_model *m, int n, const float *feat, const float *target, int epochs, int batch,
                         float lr, uint64_t seed, float *final_loss, void *stream);
/* BF16 inference for n feature rows (DEVICE): pred = predicted log(1 + k)
 * (DEVICE, n floats); r (DEVICE, n ints, may be NULL) = the sample width
 * covering k + oversample, rounded up to a multiple of 8, within [16, rmax].
 * Asynchronous. */
int hss_rank_model_predict(hss_rank_model *m, int n, const float *feat, int oversample, int rmax, float *pred,
                           int *r, void *stream);
/* Per-front record of a factorization (HOST arrays of at least cap entries,
 * any may be NULL): box id, largest node rank, final sample width, sampling
 * rounds; fronts with a single-node HSS tree (not compressed) report r = 0.
 * Returns the number of records (all fronts with |B| > 0), -1 for a null handle. */
int hss_factor_export_log(const hss_factor_t *f, int cap, int *box, int *kmax, int *r, int *rounds);

/* ---- ILU(0): the comparison preconditioner of Sec. 5 ("a standard ILU
 * preconditioner"; the variant is not named there).  Block ILU(0) on the BSR
 * pattern of A in the natural element order: L block unit lower triangular on
 * A's strictly lower pattern, U block upper triangular on A's upper pattern,
 * (L U)_ij = A_ij at every stored block, fill elsewhere dropped.  Since every
 * stored block is dense this equals scalar ILU(0) on A's scalar pattern.
 *
 * ilu0_factor: FP64, level-scheduled (a block row's level is one more than the
 * highest level of the rows it depends on; one launch per level, one CTA per
 * row).  Reads A's structure to the host once (synchronizes `stream`); does
 * not modify A.  bs <= 64; every block row must store its diagonal block.
 * Errors: HSS_EINVAL, HSS_ESINGULAR (a diagonal block of U is singular; the
 * block row goes to hss_last_error), HSS_ENOMEM, HSS_ECUDA.  *out receives a
 * new handle, owned by the caller until ilu0_destroy. */
int ilu0_factor(const hss_bsr *A, void *stream, hss_ilu_t **out);
/* y = U^-1 L^-1 x for nrhs columns (DEVICE, column-major, block-row order).
 * y may alias x.  Forward and backward level sweeps, captured once per handle
 * in a CUDA graph (one for nrhs = 1, one for blocks of 8).  Asynchronous. */
int ilu0_apply(const hss_ilu_t *M, int nrhs, const double *x, int ldx, double *y, int ldy, void *stream);
/* fgmres_solve with ILU(0) as the right preconditioner (same options,
 * statistics, errors and synchronization as fgmres_solve). */
int fgmres_solve_ilu0(const hss_bsr *A, const hss_ilu_t *M, int nrhs, const double *b, int ldb, double *x,
                      int ldx, const fgmres_opts *opts, fgmres_stats *stats, void *stream);
void ilu0_destroy(hss_ilu_t *M);

/* The apply's work split of a factorization: per stage (deepest level first,
 * the top block last) the columns per work item of the forward and backward
 * sweeps (HOST arrays of at least cap entries, either may be NULL).  Returns
 * the number of stages, or a negative error code. */
int hss_factor_apply_plan(const hss_factor_t *f, int cap, int *chunk_fwd, int *chunk_bwd);

/* Convergence history of the last fgmres_solve on this thread: Arnoldi residual
 * estimates |g_{j+1}|/||b|| of right-hand side `rhs` (HOST, up to cap values);
 * returns the count. */
int fgmres_history(int rhs, double *hist, int cap);

/* Diagnostics (no counterpart in the paper).
 * hss_launch_count: number of CUDA kernels the library has launched since it
 * was loaded (all threads).
 * hss_profile_enable(1) brackets every subsequent launch with two CUDA events
 * on its stream, grouped by kernel class; hss_profile_enable(0) stops.  Both
 * modes 1 and 2 also time named sections of the library's host code (classes
 * "host:<section>", host wall time in ms, entries in place of launches; nested
 * sections each count their inclusive time); mode 2 records those only, with
 * no events, so the host path runs as it does unprofiled.
 * hss_profile_read(-1, ...) returns the number of classes; for idx >= 0 it
 * fills the class name (HOST buffer of cap bytes), the summed event time in
 * ms, the launch count and the algorithmic work the library attributes to
 * those launches (flops for GEMM classes, bytes for apply/SpMV classes, 0 when
 * not tracked).  Reading synchronizes the pending events.
 * hss_profile_reset clears the classes.
 * hss_alloc_count: number of memory requests the library has served since it
 * was loaded (all threads): every device allocation (cudaMalloc), every
 * chunk or pinned staging buffer taken from its scratch pool, every piece of
 * call scratch (device bump allocation or upload staging).  A call that
 * leaves it unchanged allocated nothing.
 * hss_tc_timeout_selftest: runs one tile of the tensor-core GEMM kernel on an
 * internal 128 x 128 x 32 problem with the MMAs left out, so its bounded
 * mbarrier wait expires after spin_limit polls (1 .. 2^26); returns
 * HSS_ETIMEOUT when the kernel reported the expiry (the expected result),
 * with nothing left in flight and the context usable.  Test hook. */
long hss_launch_count(void);
long hss_alloc_count(void);
/* The GEMM engine tuner's process-wide choices (tensor_cores = 3): with
 * idx < 0 the number of shape classes timed so far; otherwise class idx (in
 * the order they were timed): its key (bits 0-11 log2 k, 12-23 log2 n, 24-35
 * log2 m, rounded up; bit 38 generated B, 39 transposed A; bits 40-47 the
 * tensor-core kernel timed, 1 = TMA-fed; bits 48+ device),
 * the engine kept (0 SIMT, else the tensor-core kernel) and both times (ms,
 * one problem alone on a scratch C).  Returns HSS_OK or -HSS_EINVAL. */
int hss_gemm_tuner_read(int idx, long long *key, int *engine, float *ms_simt, float *ms_tc);
int hss_tc_timeout_selftest(long spin_limit, void *stream);
int hss_profile_enable(int on);
int hss_profile_reset(void);
int hss_profile_read(int idx, char *name, int cap, double *total_ms, long *launches, double *work);

void hss_tree_destroy(hss_tree *t);
void hss_factor_destroy(hss_factor_t *f);
const char *hss_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HSSND_H */
