"""Nested-dissection box tree and interior/boundary dof sets (paper Sec. 4.0).

Definitions followed:
  * The dofs are split recursively into pairs of sibling boxes; there is no
    single root box (the tree is a forest of two level-1 boxes, footnote of
    Sec. 4.0).  Refinement stops when a box holds few enough dofs for dense
    linear algebra (Sec. 4.2: m = N / 2^L).
  * For a box sigma, a dof is a boundary dof (B^sigma) when the matrix couples
    it to a dof outside sigma, and an interior dof (I^sigma) otherwise
    (connectivity graph (1) of Sec. 4.0).  Coupling is structural: a stored
    block of the block-sparse A couples every dof pair it covers.
  * For a parent sigma of the sibling pair {mu, nu} the remaining interior and
    boundary sets are I^ = (B^mu u B^nu) n I^sigma and B^ = (B^mu u B^nu) n B^sigma
    (Sec. 4.1); B^ equals B^sigma.
  * Elimination order: leaf interiors first, then the I^ sets level by level
    towards the top, then B^1, B^2 (eq. (31)).

Readings where the paper is silent (Fig. 4/5 only show pictures):
  * cut direction: the axis with the most elements, ties to the last axis
    (y in 2D, z in 3D; the level-1 cut of the paper's box scheme is horizontal);
    'hslab' always cuts the last axis and 'vslab' the first, while they can;
  * the lower-coordinate child gets floor(n/2) elements and is child 0;
  * a box is a leaf when it holds <= leaf_max dofs or a single element;
  * boxes are numbered breadth first; dofs inside every set are ordered by a
    depth-first walk of the leaves (child 0 first, ascending global dof id
    inside a leaf); a parent front is ordered [I^ ; B^].
"""
from collections import deque

import numpy as np


def _split_axis(ext, dim, scheme):
    if scheme == "hslab" and ext[dim - 1] > 1:
        return dim - 1
    if scheme == "vslab" and ext[0] > 1:
        return 0
    best = 0
    for a in range(dim):
        if ext[a] >= ext[best]:
            best = a
    return best


def nd_order(dim, n, p, row_ptr, col_idx, leaf_max=64, scheme="box"):
    """Return a dict describing the box tree, the I/B sets and the orderings.

    dim, n[0..dim), p: structured element grid (element e = ix + nx*(iy + ny*iz));
    row_ptr, col_idx: block-sparse structure, one block row per element.
    """
    n = [int(v) for v in n[:dim]] + [1] * (3 - dim)
    bs = (p + 1) ** dim
    ne = n[0] * n[1] * n[2]
    if ne < 2:
        raise ValueError("need at least two elements")
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)

    # ---- box tree, breadth first -------------------------------------
    lo, hi, level, parent, child = [], [], [], [], []

    def nel(l, h):
        return (h[0] - l[0]) * (h[1] - l[1]) * (h[2] - l[2])

    def split(l, h):
        ext = [h[a] - l[a] for a in range(3)]
        ax = _split_axis(ext, dim, scheme)
        mid = l[ax] + ext[ax] // 2
        h0 = list(h); h0[ax] = mid
        l1 = list(l); l1[ax] = mid
        return (list(l), h0), (l1, list(h))

    q = deque()
    for (l, h) in split([0, 0, 0], n):
        q.append((l, h, 1, -1))
    while q:
        l, h, lev, par = q.popleft()
        b = len(lo)
        lo.append(l); hi.append(h); level.append(lev); parent.append(par); child.append([-1, -1])
        if par >= 0:
            child[par][0 if child[par][0] < 0 else 1] = b
        if not (nel(l, h) * bs <= leaf_max or nel(l, h) == 1):
            for (cl, ch) in split(l, h):
                q.append((cl, ch, lev + 1, b))
    nbox = len(lo)
    lo = np.array(lo, dtype=np.int64); hi = np.array(hi, dtype=np.int64)
    level = np.array(level, dtype=np.int64); parent = np.array(parent, dtype=np.int64)
    child = np.array(child, dtype=np.int64)
    is_leaf = child[:, 0] < 0
    nelem_box = np.prod(hi - lo, axis=1)

    # ---- depth-first dof positions -----------------------------------
    pos0 = np.zeros(nbox, dtype=np.int64)
    pos1 = np.zeros(nbox, dtype=np.int64)

    def assign(b, start):
        pos0[b] = start
        pos1[b] = start + nelem_box[b] * bs
        if not is_leaf[b]:
            c0, c1 = child[b]
            assign(c0, start)
            assign(c1, start + nelem_box[c0] * bs)

    assign(0, 0)
    assign(1, nelem_box[0] * bs)

    dfs_dof = np.empty(ne * bs, dtype=np.int64)      # DFS position -> global dof
    elem_leaf = np.empty(ne, dtype=np.int64)
    for b in np.nonzero(is_leaf)[0]:
        p0 = pos0[b]
        k = 0
        for iz in range(lo[b, 2], hi[b, 2]):
            for iy in range(lo[b, 1], hi[b, 1]):
                for ix in range(lo[b, 0], hi[b, 0]):
                    e = ix + n[0] * (iy + n[1] * iz)
                    elem_leaf[e] = b
                    dfs_dof[p0 + k * bs: p0 + (k + 1) * bs] = e * bs + np.arange(bs)
                    k += 1
    maxlev = int(level.max())

    # box of every element at every level (-1 when its leaf is shallower)
    elem_box = -np.ones((ne, maxlev + 1), dtype=np.int64)
    for e in range(ne):
        b = elem_leaf[e]
        while b >= 0:
            elem_box[e, level[b]] = b
            b = parent[b]

    # ---- boundary flags: element e is boundary at level l when a stored block
    # (e, f) or (f, e) has f outside e's level-l box.
    bflag = np.zeros((ne, maxlev + 1), dtype=bool)
    for e in range(ne):
        for t in range(row_ptr[e], row_ptr[e + 1]):
            f = col_idx[t]
            for lev in range(1, maxlev + 1):
                be, bf = elem_box[e, lev], elem_box[f, lev]
                if be != bf:
                    if be >= 0:
                        bflag[e, lev] = True
                    if bf >= 0:
                        bflag[f, lev] = True

    dfs_elem = dfs_dof // bs

    iset, bset, fmap = [], [], []
    ni = np.zeros(nbox, dtype=np.int64)
    nb = np.zeros(nbox, dtype=np.int64)
    for b in range(nbox):
        rng = np.arange(pos0[b], pos1[b])
        el = dfs_elem[rng]
        inB = bflag[el, level[b]]
        B = dfs_dof[rng][inB]
        if is_leaf[b]:
            I = dfs_dof[rng][~inB]
        else:
            front = bflag[el, level[b] + 1]          # in B^child0 u B^child1
            if np.any(inB & ~front):
                raise AssertionError("B^sigma not contained in B^mu u B^nu")
            I = dfs_dof[rng][front & ~inB]
        iset.append(I); bset.append(B)
        ni[b] = I.size; nb[b] = B.size

    # position of each B^mu dof inside its parent's front [I^ ; B^]; level-1
    # boxes map into the top block [B^1 ; B^2]
    for b in range(nbox):
        if parent[b] >= 0:
            par = parent[b]
            fr = np.concatenate([iset[par], bset[par]])
        else:
            fr = np.concatenate([bset[0], bset[1]])
        where = {int(d): i for i, d in enumerate(fr)}
        fmap.append(np.array([where[int(d)] for d in bset[b]], dtype=np.int64))

    # elimination order: stages from the deepest level up, BFS id inside a stage
    order = sorted(range(nbox), key=lambda b: (-level[b], b))
    perm = np.concatenate([iset[b] for b in order] + [bset[0], bset[1]])

    ioff = np.concatenate([[0], np.cumsum(ni)]).astype(np.int64)
    boff = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
    return dict(
        dim=dim, n=n, p=p, bs=bs, nbox=nbox, maxlev=maxlev,
        lo=lo, hi=hi, level=level, parent=parent, child=child, is_leaf=is_leaf,
        pos0=pos0, pos1=pos1, dfs_dof=dfs_dof, bflag=bflag,
        ni=ni, nb=nb, ioff=ioff, boff=boff,
        iset=iset, bset=bset, fmap=fmap,
        iset_flat=np.concatenate(iset).astype(np.int64),
        bset_flat=np.concatenate(bset).astype(np.int64),
        fmap_flat=np.concatenate(fmap).astype(np.int64),
        order=np.array(order, dtype=np.int64), perm=perm,
    )
