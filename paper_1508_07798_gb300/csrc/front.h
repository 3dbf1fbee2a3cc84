// Device-side descriptors of fronts and per-stage work lists.
#pragma once
#include "internal.h"

namespace hssnd {

constexpr int PANEL_NT = 512;
constexpr int PANEL_SMALL_NT = 128;   // register panels of at most this many rows
constexpr int PANEL_KB_MAX = 32;
constexpr int PANEL_SMEM_MAX = 200 * 1024;

// One front (box) of the factorization, or the top block.
struct FrontDev {
    long foff;        // offset of the n x n column-major front matrix in the arena (elements)
    int n, ni, nb;    // n = ni + nb
    int ioff;         // offset of the front's I entries in per-I arrays (pivots, gather list)
    int iset_off;     // offset of the I dof list in the tree's iset (top block: in topset)
    int iperm_off;    // offset of the permuted I list (gather list of the apply)
    int bset_off;     // offset of the B dof list in the tree's bset
    int leaf;         // leaf front (all of A(front, front) comes from A)
    int box;          // box id (-1 for the top block)
};

// A front element of the current stage: where its dofs start inside the front.
struct StageElem {
    int elem;
    int front;        // stage-local front index
    int fpos;         // position of the element's first dof inside [I ; B]
    int side;         // which child's B it belongs to (parent fronts)
};

struct PanelJob {
    int front;        // stage-local front index
    int k0, kb;
    int rlim;         // pivots are searched among the rows (positions) below rlim only: an
                      // elimination split into phases (the structured merge) keeps each
                      // phase's pivots inside its own block of rows; ni for a plain sweep
    int smem;         // 1: panel in shared memory
    long aoff;        // offset of this job's Aold (kb x n) in the workspace
    long xoff;        // offset of the pivot-block inverse X (kb x kb)
    long moff;        // offset of the row-move list (1 + 4 * PANEL_KB_MAX ints)
};

// A tile of the post-panel work (see k_gj_post).
struct PanelTile {
    int job;
    int type;         // 0: 32 columns outside the panel; 1: 64 rows outside [k0, ni)
    int start;
    int c_lo, c_hi;   // type 0: only columns in [c_lo, c_hi) (the panel's block)
};

// The end of a block of up to PANEL_BLOCK panels of one front: the columns
// outside the block receive the block's row moves and one update of width
// `width` (see k_gj_block_post).
constexpr int PANEL_BLOCK = 8;
constexpr int PANEL_BLOCK_MIN_N = 2048;   // fronts at least this large run in blocks
struct BlockJob {
    int front;        // stage-local front index
    int k0, width;    // block columns [k0, k0 + width)
    int np;           // panels in the block
    int job[PANEL_BLOCK];   // their panel jobs (move lists)
    long aoff;        // offset of this block's Aold (width x n) in the workspace
};
struct BlockTile {
    int bjob;
    int start;        // first of 32 columns
};

template <class T>
int launch_scatter_A(const hss_bsr *A, const StageElem *se, int nse, int *elem_slot, const FrontDev *fr, T *arena,
                     cudaStream_t s);
template <class T>
int launch_gj_panel(const PanelJob *jobs, int njobs, size_t smem, const FrontDev *fr, T *arena, T *xws, int *mws,
                    int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s,
                    double flops = 0.0);
template <class T>
int launch_gj_panel_reg(const PanelJob *jobs, int njobs, int kb, int rows, const FrontDev *fr, T *arena, T *xws,
                        int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s,
                        double flops = 0.0);
bool panel_reg_fits(int kb, int rows, int tsize);
// Cluster-resident panel (k_gj_panel_cl): rows spread over a cluster of 2..16
// CTAs; for kb = PANEL_KB_MAX and panels too tall for one CTA's registers.
bool panel_cl_fits(int kb, int rows, int tsize);
// rows a cluster panel of `rows` rows is launched for (its shape's capacity);
// jobs of one launch share it
int panel_cl_capacity(int rows, int tsize);
constexpr int PANEL_CL_MIN_NI = 6144;   // fronts with more interior dofs take the cluster panel
template <class T>
int launch_gj_panel_cl(const PanelJob *jobs, int njobs, int cap, size_t smem, const FrontDev *fr, T *arena, T *xws,
                       int *mws, int *piv, int *rperm, const int *ilist, int *iperm, int *status, cudaStream_t s,
                       double flops = 0.0);
template <class T>
int launch_gj_block_post(const BlockTile *tiles, int ntiles, const BlockJob *bjobs, const PanelJob *jobs,
                         const FrontDev *fr, T *arena, T *aold, const int *mws, cudaStream_t s);
template <class T>
int launch_gj_post(const PanelTile *tiles, int ntiles, const PanelJob *jobs, const FrontDev *fr, T *arena, T *aold,
                   const T *xws, const int *mws, cudaStream_t s);

}  // namespace hssnd
