// nd_order: nested-dissection box tree and interior/boundary dof sets
// (paper Sec. 4.0, graph (1); Sec. 4.1 remaining sets I^ and B^; eq. (31)).
//
// Host: box geometry (recursive bisection of element ranges, breadth-first
// numbering).  Device: per-element ancestor boxes, boundary flags from the
// block-sparse structure, per-box compaction of the I/B sets and of the
// child-to-parent front maps.
#include <algorithm>
#include <deque>

#include "internal.h"
#include "prof.h"

namespace hssnd {

struct BoxGeom {
    int lo[3], hi[3];
    int level, parent, child0, child1;
};

static long box_nel(const BoxGeom &b) {
    return (long)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}

// Cut axis: 'box' takes the axis with the most elements, ties to the last
// axis; slabs cut their axis while it has more than one element.
static int split_axis(const int ext[3], int dim, int scheme) {
    if (scheme == HSS_SCHEME_HSLAB && ext[dim - 1] > 1) return dim - 1;
    if (scheme == HSS_SCHEME_VSLAB && ext[0] > 1) return 0;
    int best = 0;
    for (int a = 0; a < dim; ++a)
        if (ext[a] >= ext[best]) best = a;
    return best;
}

static void split_box(const int lo[3], const int hi[3], int dim, int scheme, BoxGeom &c0, BoxGeom &c1) {
    int ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int ax = split_axis(ext, dim, scheme);
    int mid = lo[ax] + ext[ax] / 2;
    for (int a = 0; a < 3; ++a) {
        c0.lo[a] = lo[a]; c0.hi[a] = hi[a];
        c1.lo[a] = lo[a]; c1.hi[a] = hi[a];
    }
    c0.hi[ax] = mid;
    c1.lo[ax] = mid;
}

// ---------------------------------------------------------------- kernels
struct NdBoxDev {
    int lo[3], hi[3];
    int level, parent, child0, child1, pos0e, pos1e;  // DFS element range [pos0e, pos1e)
};

__global__ void k_nd_ancestors(const NdBoxDev *__restrict__ box, int nx, int ny, int nelem, int maxlev,
                               int *__restrict__ anc, int *__restrict__ dfs_elem) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nelem) return;
    int ix = e % nx, iy = (e / nx) % ny, iz = e / (nx * ny);
    int c[3] = {ix, iy, iz};
    for (int l = 0; l <= maxlev; ++l) anc[(long)e * (maxlev + 1) + l] = -1;
    auto inside = [&](int b) {
        const NdBoxDev &B = box[b];
        return c[0] >= B.lo[0] && c[0] < B.hi[0] && c[1] >= B.lo[1] && c[1] < B.hi[1] && c[2] >= B.lo[2] &&
               c[2] < B.hi[2];
    };
    int b = inside(0) ? 0 : 1;
    while (true) {
        anc[(long)e * (maxlev + 1) + box[b].level] = b;
        if (box[b].child0 < 0) break;
        b = inside(box[b].child0) ? box[b].child0 : box[b].child1;
    }
    const NdBoxDev &L = box[b];
    int wx = L.hi[0] - L.lo[0], wy = L.hi[1] - L.lo[1];
    int local = (ix - L.lo[0]) + wx * ((iy - L.lo[1]) + wy * (iz - L.lo[2]));
    dfs_elem[L.pos0e + local] = e;
}

// Element e is boundary at level l when a stored block (e,f) or (f,e) has f
// outside e's level-l box (bit l of flag[e]).
__global__ void k_nd_flags(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, int nelem, int maxlev,
                           const int *__restrict__ anc, unsigned *__restrict__ flag, int *__restrict__ err) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nelem) return;
    unsigned mine = 0;
    const int *ae = anc + (long)e * (maxlev + 1);
    for (int t = row_ptr[e]; t < row_ptr[e + 1]; ++t) {
        int f = col_idx[t];
        if (f < 0 || f >= nelem) {
            atomicExch(err, 1);
            continue;
        }
        if (f == e) continue;
        const int *af = anc + (long)f * (maxlev + 1);
        unsigned other = 0;
        for (int l = 1; l <= maxlev; ++l) {
            if (ae[l] != af[l]) {
                if (ae[l] >= 0) mine |= 1u << l;
                if (af[l] >= 0) other |= 1u << l;
            }
        }
        if (other) atomicOr(&flag[f], other);
    }
    if (mine) atomicOr(&flag[e], mine);
}

template <int NT> __device__ int block_excl_scan(int v, int *total, int *sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < NT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) sh[lane] = s;
    }
    __syncthreads();
    int before = (w > 0 ? sh[w - 1] : 0) + x - v;
    *total = sh[NT / 32 - 1];
    __syncthreads();
    return before;
}

constexpr int ND_NT = 256;

// Per box: element counts of B (bit level) and I (leaf: not B; internal: in
// B^child0 u B^child1 = bit level+1, not B).
__global__ void k_nd_count(const NdBoxDev *__restrict__ box, const int *__restrict__ dfs_elem,
                           const unsigned *__restrict__ flag, int *__restrict__ cntB, int *__restrict__ cntI) {
    int b = blockIdx.x;
    const NdBoxDev B = box[b];
    bool leaf = B.child0 < 0;
    int nb = 0, ni = 0;
    for (int q = B.pos0e + threadIdx.x; q < B.pos1e; q += ND_NT) {
        unsigned f = flag[dfs_elem[q]];
        bool inB = (f >> B.level) & 1u;
        bool inF = leaf ? true : ((f >> (B.level + 1)) & 1u);
        nb += inB;
        ni += (!inB && inF);
    }
    for (int o = 16; o > 0; o >>= 1) {
        nb += __shfl_down_sync(0xffffffffu, nb, o);
        ni += __shfl_down_sync(0xffffffffu, ni, o);
    }
    __shared__ int sb[ND_NT / 32], si[ND_NT / 32];
    if ((threadIdx.x & 31) == 0) {
        sb[threadIdx.x >> 5] = nb;
        si[threadIdx.x >> 5] = ni;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tb = 0, ti = 0;
        for (int w = 0; w < ND_NT / 32; ++w) {
            tb += sb[w];
            ti += si[w];
        }
        cntB[b] = tb;
        cntI[b] = ti;
    }
}

// Per box: write its I and B dof lists (depth-first order) and, for an
// internal box, the position of every child-B dof inside this box's front
// [I^ ; B^].  Level-1 boxes map into the top block [B^1 ; B^2].
__global__ void k_nd_emit(const NdBoxDev *__restrict__ box, const int *__restrict__ dfs_elem,
                          const unsigned *__restrict__ flag, int bs, const int *__restrict__ ioff,
                          const int *__restrict__ boff, const int *__restrict__ nI, const int *__restrict__ nB,
                          int *__restrict__ iset, int *__restrict__ bset, int *__restrict__ fmap) {
    __shared__ int sh[ND_NT / 32];
    int b = blockIdx.x;
    const NdBoxDev B = box[b];
    bool leaf = B.child0 < 0;
    if (B.level == 1) {
        int base = (b == 1) ? nB[0] : 0;
        for (int i = threadIdx.x; i < nB[b]; i += ND_NT) fmap[boff[b] + i] = base + i;
    }
    int split = leaf ? B.pos1e : box[B.child0].pos0e + (box[B.child0].pos1e - box[B.child0].pos0e);
    int nfront0 = leaf ? 0 : nB[B.child0] / bs;
    int carryB = 0, carryI = 0, carryF = 0;
    for (int q0 = B.pos0e; q0 < B.pos1e; q0 += ND_NT) {
        int q = q0 + threadIdx.x;
        bool valid = q < B.pos1e;
        int e = valid ? dfs_elem[q] : 0;
        unsigned f = valid ? flag[e] : 0u;
        bool inB = valid && ((f >> B.level) & 1u);
        bool inF = valid && (leaf ? true : ((f >> (B.level + 1)) & 1u));
        bool inI = inF && !inB;
        int tB, tI, tF;
        int rB = block_excl_scan<ND_NT>(inB ? 1 : 0, &tB, sh) + carryB;
        int rI = block_excl_scan<ND_NT>(inI ? 1 : 0, &tI, sh) + carryI;
        int rF = block_excl_scan<ND_NT>((!leaf && inF) ? 1 : 0, &tF, sh) + carryF;
        if (inB)
            for (int j = 0; j < bs; ++j) bset[boff[b] + rB * bs + j] = e * bs + j;
        if (inI)
            for (int j = 0; j < bs; ++j) iset[ioff[b] + rI * bs + j] = e * bs + j;
        if (!leaf && inF) {
            int side = q < split ? 0 : 1;
            int child = side ? B.child1 : B.child0;
            int idx = rF - (side ? nfront0 : 0);
            int target = inB ? (nI[b] / bs + rB) : rI;  // element slot inside the front
            for (int j = 0; j < bs; ++j) fmap[boff[child] + idx * bs + j] = target * bs + j;
        }
        carryB += tB;
        carryI += tI;
        carryF += tF;
    }
}

// ---------------------------------------------------------------- host
// HSS tree over the dofs `dofs` (ascending depth-first positions, e.g. B^box
// or a subset of it) from the nested-dissection subtree of `box`: a node per
// box of the subtree that holds some of the dofs, empty boxes removed and
// single-child chains collapsed; nodes in post-order, root last.
void hss_nodes_over(const hss_tree *t, const std::vector<int> &elem_pos, int box, const std::vector<int> &dofs,
                    std::vector<HssNode> &nodes) {
    nodes.clear();
    if (dofs.empty()) return;
    std::vector<long> pos(dofs.size());
    for (size_t i = 0; i < dofs.size(); ++i) pos[i] = (long)elem_pos[dofs[i] / t->bs] * t->bs + dofs[i] % t->bs;
    struct Rec {
        const hss_tree *t;
        std::vector<long> &pos;
        std::vector<HssNode> &nodes;
        int go(int bx) {
            long p0 = t->pos0[bx], p1 = t->pos1[bx];
            int lo = (int)(std::lower_bound(pos.begin(), pos.end(), p0) - pos.begin());
            int hi = (int)(std::lower_bound(pos.begin(), pos.end(), p1) - pos.begin());
            if (hi == lo) return -1;
            if (t->child0[bx] < 0) {
                nodes.push_back({lo, hi, -1, -1, 0});
                return (int)nodes.size() - 1;
            }
            int c0 = go(t->child0[bx]);
            int c1 = go(t->child1[bx]);
            if (c0 < 0) return c1;
            if (c1 < 0) return c0;
            nodes.push_back({lo, hi, c0, c1, 0});
            return (int)nodes.size() - 1;
        }
    } rec{t, pos, nodes};
    rec.go(box);
    int root = (int)nodes.size() - 1;
    nodes[root].depth = 0;
    for (int i = root; i >= 0; --i)
        if (nodes[i].a >= 0) {
            nodes[nodes[i].a].depth = nodes[i].depth + 1;
            nodes[nodes[i].b].depth = nodes[i].depth + 1;
        }
}

std::vector<int> elem_positions(const hss_tree *t) {
    std::vector<int> elem_pos(t->nelem);
    for (int q = 0; q < t->nelem; ++q) elem_pos[t->dfs_elem[q]] = q;
    return elem_pos;
}

static void build_hss_trees(hss_tree *t) {
    const std::vector<int> elem_pos = elem_positions(t);
    t->hss.assign(t->nbox, {});
    for (int b = 0; b < t->nbox; ++b) {
        if (t->nb[b] == 0) continue;
        std::vector<int> dofs(t->bset.begin() + t->boff[b], t->bset.begin() + t->boff[b + 1]);
        hss_nodes_over(t, elem_pos, b, dofs, t->hss[b]);
    }
}

}  // namespace hssnd

using namespace hssnd;

extern "C" int nd_order(const hss_mesh *mesh, const hss_bsr *A, const hss_nd_opts *opts, void *stream,
                        hss_tree **out) {
    if (!mesh || !A || !out) {
        set_error("nd_order: null argument");
        return HSS_EINVAL;
    }
    *out = nullptr;
    hss_nd_opts o;
    hss_nd_opts_default(&o);
    if (opts) o = *opts;
    int dim = mesh->dim, p = mesh->p;
    if (dim < 2 || dim > 3 || p < 1 || o.leaf_max < 1) {
        set_error("nd_order: need dim 2 or 3, p >= 1, leaf_max >= 1");
        return HSS_EINVAL;
    }
    int n[3] = {mesh->n[0], mesh->n[1], dim == 3 ? mesh->n[2] : 1};
    long nelem = (long)n[0] * n[1] * n[2];
    int bs = 1;
    for (int k = 0; k < dim; ++k) bs *= (p + 1);
    if (n[0] < 1 || n[1] < 1 || n[2] < 1 || nelem < 2 || A->nb != nelem || A->bs != bs || !A->row_ptr ||
        !A->col_idx) {
        set_error("nd_order: mesh and block matrix disagree (need nb = #elements >= 2, bs = (p+1)^dim)");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;

    // ---- box geometry, breadth first
    std::vector<BoxGeom> boxes;
    std::deque<BoxGeom> q;
    {
        int lo0[3] = {0, 0, 0};
        BoxGeom c0, c1;
        split_box(lo0, n, dim, o.scheme, c0, c1);
        c0.level = c1.level = 1;
        c0.parent = c1.parent = -1;
        q.push_back(c0);
        q.push_back(c1);
    }
    while (!q.empty()) {
        BoxGeom g = q.front();
        q.pop_front();
        g.child0 = g.child1 = -1;
        int id = (int)boxes.size();
        if (g.parent >= 0) {
            if (boxes[g.parent].child0 < 0)
                boxes[g.parent].child0 = id;
            else
                boxes[g.parent].child1 = id;
        }
        boxes.push_back(g);
        long ne = box_nel(g);
        if (!(ne * bs <= o.leaf_max || ne == 1)) {
            BoxGeom c0, c1;
            split_box(g.lo, g.hi, dim, o.scheme, c0, c1);
            c0.level = c1.level = g.level + 1;
            c0.parent = c1.parent = id;
            q.push_back(c0);
            q.push_back(c1);
        }
    }
    int nbox = (int)boxes.size();
    int maxlev = 0;
    for (auto &g : boxes) maxlev = std::max(maxlev, g.level);
    if (maxlev > 30) {
        set_error("nd_order: tree deeper than 30 levels");
        return HSS_EINVAL;
    }

    hss_tree *t = new hss_tree();
    t->dim = dim;
    t->n[0] = n[0]; t->n[1] = n[1]; t->n[2] = n[2];
    t->p = p;
    t->bs = bs;
    t->nelem = (int)nelem;
    t->ndof = (int)(nelem * bs);
    t->nbox = nbox;
    t->maxlev = maxlev;
    t->opts = o;
    t->level.resize(nbox); t->parent.resize(nbox); t->child0.resize(nbox); t->child1.resize(nbox);
    t->lohi.resize(6 * nbox); t->pos0.resize(nbox); t->pos1.resize(nbox);
    for (int b = 0; b < nbox; ++b) {
        t->level[b] = boxes[b].level;
        t->parent[b] = boxes[b].parent;
        t->child0[b] = boxes[b].child0;
        t->child1[b] = boxes[b].child1;
        for (int a = 0; a < 3; ++a) {
            t->lohi[6 * b + a] = boxes[b].lo[a];
            t->lohi[6 * b + 3 + a] = boxes[b].hi[a];
        }
    }
    // depth-first dof ranges
    std::vector<long> p0(nbox);
    {
        // iterative DFS: child 0 first
        struct Item { int b; long start; };
        std::vector<Item> st = {{1, box_nel(boxes[0]) * bs}, {0, 0}};
        while (!st.empty()) {
            Item it = st.back();
            st.pop_back();
            p0[it.b] = it.start;
            t->pos0[it.b] = (int)it.start;
            t->pos1[it.b] = (int)(it.start + box_nel(boxes[it.b]) * bs);
            if (boxes[it.b].child0 >= 0) {
                int c0 = boxes[it.b].child0, c1 = boxes[it.b].child1;
                st.push_back({c1, it.start + box_nel(boxes[c0]) * bs});
                st.push_back({c0, it.start});
            }
        }
    }
    std::vector<NdBoxDev> hb(nbox);
    for (int b = 0; b < nbox; ++b) {
        for (int a = 0; a < 3; ++a) {
            hb[b].lo[a] = boxes[b].lo[a];
            hb[b].hi[a] = boxes[b].hi[a];
        }
        hb[b].level = boxes[b].level;
        hb[b].parent = boxes[b].parent;
        hb[b].child0 = boxes[b].child0;
        hb[b].child1 = boxes[b].child1;
        hb[b].pos0e = t->pos0[b] / bs;
        hb[b].pos1e = t->pos1[b] / bs;
    }

    // call scratch (returned to the scratch cache when W goes out of scope)
    Work W(s);
    ScratchPtr d_box, d_anc, d_dfs, d_flag, d_err, d_cnt, d_off;
    int rc;
    if ((rc = W.stage_bytes(hb.data(), sizeof(NdBoxDev) * hb.size(), &d_box.p)) ||
        (rc = W.dalloc_bytes(sizeof(int) * nelem * (maxlev + 1), &d_anc.p)) ||
        (rc = W.dalloc_bytes(sizeof(int) * nelem, &d_dfs.p)) || (rc = W.dalloc_bytes(sizeof(unsigned) * nelem, &d_flag.p)) ||
        (rc = W.dalloc_bytes(sizeof(int), &d_err.p)) || (rc = W.dalloc_bytes(sizeof(int) * 2 * nbox, &d_cnt.p)) ||
        (rc = W.dalloc_bytes(sizeof(int) * 4 * nbox, &d_off.p))) {
        delete t;
        return rc;
    }
    auto fail = [&](int code) {
        delete t;
        return code;
    };
    if (cudaMemsetAsync(d_flag.p, 0, sizeof(unsigned) * nelem, s) != cudaSuccess ||
        cudaMemsetAsync(d_err.p, 0, sizeof(int), s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "nd_order memset"));
    int nt = 256;
    { HSS_PROF("nd_ancestors", s);
    k_nd_ancestors<<<cdiv(nelem, nt), nt, 0, s>>>(d_box.as<NdBoxDev>(), n[0], n[1], (int)nelem, maxlev,
                                                   d_anc.as<int>(), d_dfs.as<int>()); }
    { HSS_PROF("nd_flags", s);
    k_nd_flags<<<cdiv(nelem, nt), nt, 0, s>>>(A->row_ptr, A->col_idx, (int)nelem, maxlev, d_anc.as<int>(),
                                               d_flag.as<unsigned>(), d_err.as<int>()); }
    int *cntB = d_cnt.as<int>(), *cntI = cntB + nbox;
    { HSS_PROF("nd_count", s);
    k_nd_count<<<nbox, ND_NT, 0, s>>>(d_box.as<NdBoxDev>(), d_dfs.as<int>(), d_flag.as<unsigned>(), cntB, cntI); }
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(cuda_fail(e, "nd_order kernels"));
    }
    std::vector<int> hc(2 * nbox);
    int herr = 0;
    if (cudaMemcpyAsync(hc.data(), d_cnt.p, sizeof(int) * 2 * nbox, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "nd_order count readback"));
    if (herr) {
        set_error("nd_order: column index out of range in the block matrix");
        return fail(HSS_EINVAL);
    }
    t->ni.resize(nbox); t->nb.resize(nbox); t->ioff.resize(nbox + 1); t->boff.resize(nbox + 1);
    t->ioff[0] = t->boff[0] = 0;
    for (int b = 0; b < nbox; ++b) {
        t->nb[b] = hc[b] * bs;
        t->ni[b] = hc[nbox + b] * bs;
        t->ioff[b + 1] = t->ioff[b] + t->ni[b];
        t->boff[b + 1] = t->boff[b] + t->nb[b];
    }
    // offsets and sizes to the device
    std::vector<int> hoff(4 * nbox);
    for (int b = 0; b < nbox; ++b) {
        hoff[b] = t->ioff[b];
        hoff[nbox + b] = t->boff[b];
        hoff[2 * nbox + b] = t->ni[b];
        hoff[3 * nbox + b] = t->nb[b];
    }
    int ilen = t->ioff[nbox], blen = t->boff[nbox];
    if ((rc = t->d_iset.alloc(sizeof(int) * std::max(ilen, 1))) || (rc = t->d_bset.alloc(sizeof(int) * blen)) ||
        (rc = t->d_fmap.alloc(sizeof(int) * blen)))
        return fail(rc);
    if (cudaMemcpyAsync(d_off.p, hoff.data(), sizeof(int) * 4 * nbox, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "nd_order offsets"));
    int *dio = d_off.as<int>();
    { HSS_PROF("nd_emit", s);
    k_nd_emit<<<nbox, ND_NT, 0, s>>>(d_box.as<NdBoxDev>(), d_dfs.as<int>(), d_flag.as<unsigned>(), bs, dio,
                                      dio + nbox, dio + 2 * nbox, dio + 3 * nbox, t->d_iset.as<int>(),
                                      t->d_bset.as<int>(), t->d_fmap.as<int>()); }
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(cuda_fail(e, "k_nd_emit"));
    }
    t->iset.resize(ilen);
    t->bset.resize(blen);
    t->fmap.resize(blen);
    t->dfs_elem.resize(nelem);
    if ((ilen && cudaMemcpyAsync(t->iset.data(), t->d_iset.p, sizeof(int) * ilen, cudaMemcpyDeviceToHost, s)) ||
        cudaMemcpyAsync(t->bset.data(), t->d_bset.p, sizeof(int) * blen, cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(t->fmap.data(), t->d_fmap.p, sizeof(int) * blen, cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(t->dfs_elem.data(), d_dfs.p, sizeof(int) * nelem, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return fail(cuda_fail(cudaGetLastError(), "nd_order readback"));

    // stages (deepest level first) and the eq. (31) elimination order
    t->stages.clear();
    for (int lev = maxlev; lev >= 1; --lev) {
        std::vector<int> st;
        for (int b = 0; b < nbox; ++b)
            if (t->level[b] == lev) st.push_back(b);
        t->stages.push_back(st);
    }
    t->perm.clear();
    for (auto &st : t->stages)
        for (int b : st) t->perm.insert(t->perm.end(), t->iset.begin() + t->ioff[b], t->iset.begin() + t->ioff[b + 1]);
    for (int b = 0; b < 2; ++b)
        t->perm.insert(t->perm.end(), t->bset.begin() + t->boff[b], t->bset.begin() + t->boff[b + 1]);
    build_hss_trees(t);
    t->ninst = 1;
    t->inst_top = {0};
    t->inst_dof = {0, t->ndof};
    t->inst_elem = {0, t->nelem};
    t->box_inst.assign(nbox, 0);
    t->box_local.resize(nbox);
    for (int b = 0; b < nbox; ++b) t->box_local[b] = b;
    *out = t;
    return HSS_OK;
}

extern "C" int nd_order_batched(int ninst, const hss_mesh *meshes, const hss_bsr *As, const hss_nd_opts *opts,
                                void *stream, hss_tree **out) {
    if (!meshes || !As || !out || ninst < 1) {
        set_error("nd_order_batched: null argument or ninst < 1");
        return HSS_EINVAL;
    }
    *out = nullptr;
    std::vector<hss_tree *> parts(ninst, nullptr);
    auto drop = [&](int rc) {
        for (auto *q : parts) delete q;
        return rc;
    };
    for (int i = 0; i < ninst; ++i) {
        int rc = nd_order(meshes + i, As + i, opts, stream, &parts[i]);
        if (rc) {
            set_error("nd_order_batched: instance " + std::to_string(i) + ": " + hss_last_error());
            return drop(rc);
        }
        if (parts[i]->bs != parts[0]->bs) {
            set_error("nd_order_batched: instances must share the block size (instance " + std::to_string(i) + ")");
            return drop(HSS_EINVAL);
        }
    }
    hss_tree *F = new hss_tree;
    const hss_tree &P0 = *parts[0];
    F->dim = P0.dim;
    std::copy(P0.n, P0.n + 3, F->n);
    F->p = P0.p;
    F->bs = P0.bs;
    F->opts = P0.opts;
    F->ninst = ninst;
    F->ioff.push_back(0);
    F->boff.push_back(0);
    int dof0 = 0, elem0 = 0, box0 = 0;
    for (int i = 0; i < ninst; ++i) {
        const hss_tree &P = *parts[i];
        const int ib = (int)F->iset.size(), bb = (int)F->bset.size();
        F->inst_top.push_back(box0);
        F->inst_dof.push_back(dof0);
        F->inst_elem.push_back(elem0);
        F->maxlev = std::max(F->maxlev, P.maxlev);
        for (int b = 0; b < P.nbox; ++b) {
            F->level.push_back(P.level[b]);
            F->parent.push_back(P.parent[b] < 0 ? -1 : P.parent[b] + box0);
            F->child0.push_back(P.child0[b] < 0 ? -1 : P.child0[b] + box0);
            F->child1.push_back(P.child1[b] < 0 ? -1 : P.child1[b] + box0);
            F->lohi.insert(F->lohi.end(), P.lohi.begin() + 6 * b, P.lohi.begin() + 6 * b + 6);
            F->pos0.push_back(P.pos0[b] + dof0);
            F->pos1.push_back(P.pos1[b] + dof0);
            F->ni.push_back(P.ni[b]);
            F->nb.push_back(P.nb[b]);
            F->ioff.push_back(ib + P.ioff[b + 1]);
            F->boff.push_back(bb + P.boff[b + 1]);
            F->hss.push_back(P.hss[b]);
            F->box_inst.push_back(i);
            F->box_local.push_back(b);
        }
        for (int v : P.iset) F->iset.push_back(v + dof0);
        for (int v : P.bset) F->bset.push_back(v + dof0);
        F->fmap.insert(F->fmap.end(), P.fmap.begin(), P.fmap.end());
        for (int v : P.perm) F->perm.push_back(v + dof0);
        for (int v : P.dfs_elem) F->dfs_elem.push_back(v + elem0);
        dof0 += P.ndof;
        elem0 += P.nelem;
        box0 += P.nbox;
    }
    F->inst_dof.push_back(dof0);
    F->inst_elem.push_back(elem0);
    F->ndof = dof0;
    F->nelem = elem0;
    F->nbox = box0;
    for (int lev = F->maxlev; lev >= 1; --lev) {
        std::vector<int> st;
        for (int b = 0; b < F->nbox; ++b)
            if (F->level[b] == lev) st.push_back(b);
        F->stages.push_back(st);
    }
    drop(0);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = upload(F->d_iset, F->iset.empty() ? std::vector<int>{0} : F->iset, s)) ||
        (rc = upload(F->d_bset, F->bset, s)) || (rc = upload(F->d_fmap, F->fmap, s))) {
        delete F;
        return rc;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        delete F;
        return cuda_fail(cudaGetLastError(), "nd_order_batched upload");
    }
    *out = F;
    return HSS_OK;
}

extern "C" int hss_tree_info(const hss_tree *t, hss_tree_desc *d) {
    if (!t || !d) {
        set_error("hss_tree_info: null argument");
        return HSS_EINVAL;
    }
    d->ndof = t->ndof;
    d->nbox = t->nbox;
    d->maxlev = t->maxlev;
    d->iset_len = t->ioff[t->nbox];
    d->bset_len = t->boff[t->nbox];
    d->bs = t->bs;
    return HSS_OK;
}

extern "C" int hss_tree_export(const hss_tree *t, int *level, int *parent, int *child0, int *child1, int *ni,
                               int *nb, int *ioff, int *boff, int *lohi, int *iset, int *bset, int *fmap,
                               int *perm) {
    if (!t) {
        set_error("hss_tree_export: null tree");
        return HSS_EINVAL;
    }
    auto cp = [](int *dst, const std::vector<int> &v, size_t n) {
        if (dst && n) std::copy(v.begin(), v.begin() + n, dst);
    };
    size_t nb_ = t->nbox;
    cp(level, t->level, nb_);
    cp(parent, t->parent, nb_);
    cp(child0, t->child0, nb_);
    cp(child1, t->child1, nb_);
    cp(ni, t->ni, nb_);
    cp(nb, t->nb, nb_);
    cp(ioff, t->ioff, nb_);
    cp(boff, t->boff, nb_);
    cp(lohi, t->lohi, 6 * nb_);
    cp(iset, t->iset, t->iset.size());
    cp(bset, t->bset, t->bset.size());
    cp(fmap, t->fmap, t->fmap.size());
    cp(perm, t->perm, t->perm.size());
    return HSS_OK;
}

extern "C" void hss_tree_destroy(hss_tree *t) { delete t; }
