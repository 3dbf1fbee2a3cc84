// Device descriptors of the randomized HSS construction (Theorem 1).
#pragma once
#include "internal.h"

namespace hssnd {

constexpr int ID_NT = 256;
constexpr int ID_MAX_SWAPS = 64;
constexpr int EXP_TILE = 32;

// Leading dimension of the ID's r x m sample block in shared memory: columns
// start on 16-byte boundaries and lda * esize / 16 is odd, so the 16-byte
// accesses of eight threads to eight columns fall in distinct banks.
__host__ __device__ inline int id_lda(int r, int esize) {
    const int q = 16 / esize;                      // values per 16 bytes
    int l = (r + q - 1) / q;                       // 16-byte units per column
    if ((l & 1) == 0) ++l;
    return l * q;
}
// Shared memory of one ID CTA: the sample block (lda x mcap), v (r), the
// squared norms (mcap) and the column order (mcap ints).
inline size_t id_smem_bytes(int r, int mcap, int esize) {
    return (size_t)esize * ((size_t)id_lda(r, esize) * mcap + r + mcap) + sizeof(int) * (size_t)mcap + 16;
}

// A front being compressed in the current sampling round.
template <class T> struct CompFront {
    const T *S;       // Schur complement inside the front (column-major)
    long lds;         // its leading dimension (the front size)
    int nb;           // order of S
    int r;            // sample width of the current sampling round
    int box;          // front id of the test-matrix counter
    long yoff, zoff;  // samples Y = S Omega, Z = S^t Psi (nb x r, ld nb) in the sample buffer
};

// One side (0: rows / U, 1: columns / V) of one HSS node.
struct NodeSide {
    long loff;        // local samples L (m x r, ld mcap), kept for exchanges and skeleton rows
    long toff;        // T (k x (m-k), ld kcap)
    long skoff;       // skeleton samples L(J,:) (k x r, ld kcap)
    long tloff;       // compressed test matrix U^t Psi_loc / V^t Omega_loc (k x r, ld kcap)
    long ordoff;      // int: order [J ; J^c] (m)
    long skioff;      // int: skeleton S indices (k)
    long talloff;     // tall basis (|R| x k, ld |R|), filled by the expansion pass
    int mcap, kcap;
};

struct NodeDev {
    int cf;           // compressed-front index of the round
    int lo, hi;       // range inside B^box
    int a, b;         // children (round-global node indices) or -1
    NodeSide s[2];
};

// One 32 x 32 tile of the expanded approximant H written into the parent front.
struct ExpandItem {
    int type;         // 0: copy S block (leaf diagonal block / whole S); 1: U^tall_a S(J_a,K_b) V^tall_b^t
    int cf;           // compressed-front index (type 1) or front descriptor index (type 0)
    int na, nb;       // nodes (type 1)
    int r0, c0;       // tile origin inside B^box (row / column index of H)
    int rlo, rhi, clo, chi;  // row / column ranges covered by the block
};

struct ExpandFront {  // where H goes: parent front (through fmap) and the optional keep copy
    const void *S;    // Schur complement of the child front
    long lds;
    int nb;
    const int *fmap;  // position of each B dof of the child inside the parent front
    long poff;        // parent front offset in the arena
    int pn;           // parent front size
    long keep_h;      // offset of the keep copy of H (-1: none)
};

// Residual probe of an accepted approximant: one CTA per (front, 128-row
// tile, 128-column tile) accumulates the tile's share of S W and (S - H) W per
// row; a second kernel forms ||(S - H) W||_F^2 and ||S W||_F^2 per front.
constexpr int PROBE_NT = 128;    // rows (threads) and columns of a tile
constexpr int PROBE_MAX = 8;     // probe vectors at most
struct ProbeItem {
    int slot;         // probed front of the round (accumulator pair)
    int f;            // stage-local front (index into the ExpandFront array)
    int box;          // counter key of the front's random matrices
    int row0, col0;   // tile origin
    long rowacc;      // offset of the front's row sums (2 x PROBE_MAX doubles per row)
};
struct ProbeFront {
    int f;
    long rowacc;
};

template <class T>
int launch_hss_id(const NodeDev *nodes, const int *work, int nwork, const CompFront<T> *cf, T *ws, int *iws,
                  int *kout, int *front_kmax, T tol, uint64_t seed, size_t smem, cudaStream_t s);
template <class T>
int launch_hss_tall(const NodeDev *nodes, const int *work, int nwork, const int *kout, T *ws, int *iws, size_t smem,
                    cudaStream_t s);
template <class T>
int launch_hss_expand(const ExpandItem *items, int nitems, const NodeDev *nodes, const int *kout,
                      const ExpandFront *ef, const T *ws, const int *iws, T *arena, T *keep, int kmax,
                      cudaStream_t s);
template <class T>
int launch_hss_probe(const ProbeItem *items, int nitems, const ProbeFront *pf, int nfronts, const ExpandFront *ef,
                     const T *arena, uint64_t seed, int nprobe, double *rowacc, double *acc, cudaStream_t s);

}  // namespace hssnd
