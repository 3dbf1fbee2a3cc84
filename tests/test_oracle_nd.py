"""Oracle pin: the nested-dissection sets checked against their definitions
(Sec. 4.0/4.1) by brute force on tiny meshes."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg


def _pattern(A):
    """Structural pattern: a stored block couples every dof pair it covers."""
    P = np.zeros((A.n, A.n), dtype=bool)
    bs = A.bs
    for e in range(A.nb):
        for t in range(A.row_ptr[e], A.row_ptr[e + 1]):
            f = A.col_idx[t]
            P[e * bs:(e + 1) * bs, f * bs:(f + 1) * bs] = True
    return P


def _box_dofs(nd, b):
    n, bs = nd["n"], nd["bs"]
    out = []
    lo, hi = nd["lo"][b], nd["hi"][b]
    for iz, iy, ix in itertools.product(range(lo[2], hi[2]), range(lo[1], hi[1]), range(lo[0], hi[0])):
        e = ix + n[0] * (iy + n[1] * iz)
        out.extend(range(e * bs, (e + 1) * bs))
    return set(out)


CASES = [(2, (2, 2), 1, 4), (2, (3, 2), 1, 8), (2, (3, 3), 1, 8), (2, (4, 4), 2, 18),
         (2, (5, 3), 1, 8), (2, (4, 4), 3, 16), (3, (2, 2, 2), 1, 8), (3, (3, 2, 2), 1, 16),
         (2, (7, 5), 1, 12)]


@pytest.mark.parametrize("scheme", ["box", "hslab", "vslab"])
@pytest.mark.parametrize("dim,n,p,leaf", CASES)
def test_sets_match_definition(dim, n, p, leaf, scheme):
    mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
    A = dg.assemble_sipg(mesh)
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx, leaf_max=leaf, scheme=scheme)
    P = _pattern(A)
    coupled = P | P.T
    N = A.n
    # level-1 boxes partition the dofs; children partition their parent
    allb = _box_dofs(nd, 0) | _box_dofs(nd, 1)
    assert allb == set(range(N)) and not (_box_dofs(nd, 0) & _box_dofs(nd, 1))
    for b in range(nd["nbox"]):
        dofs = _box_dofs(nd, b)
        nel = len(dofs) // nd["bs"]
        if nd["is_leaf"][b]:
            assert len(dofs) <= leaf or nel == 1
        else:
            assert not (len(dofs) <= leaf or nel == 1)
            c0, c1 = nd["child"][b]
            d0, d1 = _box_dofs(nd, c0), _box_dofs(nd, c1)
            assert d0 | d1 == dofs and not (d0 & d1)
        inside = np.zeros(N, dtype=bool)
        inside[list(dofs)] = True
        # definition: boundary dof = coupled to some dof outside the box
        Bdef = {i for i in dofs if coupled[i, ~inside].any()}
        assert set(nd["bset"][b].tolist()) == Bdef
        if nd["is_leaf"][b]:
            assert set(nd["iset"][b].tolist()) == dofs - Bdef
        else:
            c0, c1 = nd["child"][b]
            agg = set(nd["bset"][c0].tolist()) | set(nd["bset"][c1].tolist())
            assert set(nd["iset"][b].tolist()) == agg - Bdef       # I^ = (B^mu u B^nu) n I^sigma
            assert Bdef <= agg                                     # B^ = B^sigma
        # fmap: position of each B dof inside the parent front / top block
        par = nd["parent"][b]
        fr = (np.concatenate([nd["iset"][par], nd["bset"][par]]) if par >= 0
              else np.concatenate([nd["bset"][0], nd["bset"][1]]))
        assert np.array_equal(fr[nd["fmap"][b]], nd["bset"][b])
    # elimination order is a permutation covering every dof once
    assert np.array_equal(np.sort(nd["perm"]), np.arange(N))


def test_interior_of_each_leaf_uncoupled_from_other_boxes():
    """Graph (1) of Sec. 4.0: interiors of distinct boxes never couple."""
    mesh = dg.Mesh(2, (8, 8, 1), 1)
    A = dg.assemble_sipg(mesh)
    nd = oracle.nd_order(2, mesh.n, 1, A.row_ptr, A.col_idx, leaf_max=16)
    P = _pattern(A)
    lev = nd["level"]
    for L in range(1, nd["maxlev"] + 1):
        bx = [b for b in range(nd["nbox"]) if lev[b] == L]
        for a in bx:
            for b in bx:
                if a == b:
                    continue
                Ia, Ib = nd["iset"][a], nd["iset"][b]
                Ba = nd["bset"][a]
                if Ia.size and Ib.size and nd["is_leaf"][a] and nd["is_leaf"][b]:
                    assert not P[np.ix_(Ia, Ib)].any()
                if Ia.size and nd["is_leaf"][a]:
                    # an interior dof only touches its own box
                    assert not P[np.ix_(Ia, nd["bset"][b])].any()
                assert Ba.size >= 0


def test_c0_shape():
    mesh, A = dg.poisson_2d(16, 1)
    nd = oracle.nd_order(2, mesh.n, 1, A.row_ptr, A.col_idx, leaf_max=64)
    assert nd["maxlev"] == 4 and int(nd["is_leaf"].sum()) == 16
    assert nd["nb"][0] + nd["nb"][1] == 128          # top block of 128 dofs
    assert nd["level"][0] == nd["level"][1] == 1
    # the level-1 cut is horizontal (tie broken towards y)
    assert nd["hi"][0][1] == 8 and nd["hi"][0][0] == 16
