"""Oracle pins for the block ILU(0) comparison preconditioner (oracle/ilu.py)."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import ilu as oilu
from paper_1508_07798_gb300 import dg_inputs as dg


def _mesh(n, p):
    return dg.Mesh(len(n), tuple(n) + (1,) * (3 - len(n)), p)


def _pattern(A):
    bs = A.bs
    P = np.zeros((A.n, A.n), bool)
    for i in range(A.nb):
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col_idx[q]
            P[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = True
    return P


@pytest.mark.parametrize("n,p,kind", [((4, 3), 1, "poisson"), ((3, 3), 2, "helm"), ((2, 2, 2), 1, "poisson")])
def test_product_equals_a_on_its_pattern(n, p, kind):
    """The defining property of ILU(0): (L U)_ij = A_ij wherever A has a
    stored block; the dropped fill makes L U differ from A elsewhere."""
    mesh = _mesh(n, p)
    kap = dg.helmholtz_kappa(n[0], p) if kind == "helm" else 0.0
    A = dg.assemble_sipg(mesh, kappa=kap)
    D = dg.bsr_to_dense(A)
    L, U = oilu.ilu0_dense_factors(oilu.ilu0(A.row_ptr, A.col_idx, A.val))
    P = _pattern(A)
    E = L @ U - D
    assert np.abs(E[P]).max() <= 1e-12 * np.abs(D).max()
    assert np.abs(E[~P]).max() > 1e-3 * np.abs(D).max()


def test_element_chain_is_exact():
    """On a 1D chain of elements A is block tridiagonal: no fill is dropped,
    ILU(0) is the exact block LU and the preconditioner is A^-1."""
    mesh = dg.Mesh(2, (7, 1, 1), 2)
    A = dg.assemble_sipg(mesh)
    X = dg.random_rhs(A.n, 2, 0)
    Z = oilu.ilu0_apply(oilu.ilu0(A.row_ptr, A.col_idx, A.val), X)
    assert np.linalg.norm(Z - np.linalg.solve(dg.bsr_to_dense(A), X)) <= 1e-12 * np.linalg.norm(Z)


def _scalar_ilu0(D, P):
    """Scalar ILU(0) (row form) on the scalar pattern P, written directly."""
    a = D.copy()
    n = a.shape[0]
    for i in range(1, n):
        for k in range(i):
            if not P[i, k]:
                continue
            a[i, k] /= a[k, k]
            for j in range(k + 1, n):
                if P[i, j]:
                    a[i, j] -= a[i, k] * a[k, j]
    return np.tril(a, -1) + np.eye(n), np.triu(a)


def test_block_form_equals_scalar_ilu0():
    mesh = _mesh((3, 3), 1)
    A = dg.assemble_sipg(mesh, c_elem=dg.cosine_field(mesh, 0), kappa=3.0)
    D = dg.bsr_to_dense(A)
    Ls, Us = _scalar_ilu0(D, _pattern(A))
    Lb, Ub = oilu.ilu0_dense_factors(oilu.ilu0(A.row_ptr, A.col_idx, A.val))
    sc = np.abs(D).max()
    # the block form keeps U's diagonal blocks whole: compare the products and the off-diagonal blocks
    assert np.abs(Lb @ Ub - Ls @ Us).max() <= 1e-12 * sc
    bs = A.bs
    for i in range(A.nb):
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col_idx[q]
            if j != i:
                blk = (slice(i * bs, (i + 1) * bs), slice(j * bs, (j + 1) * bs))
                # Lb = Ls diag(Ld)^-1 and Ub = diag(Ld) Us, Ld the unit-lower diagonal blocks of Ls
                if j < i:
                    Ld = Ls[j * bs:(j + 1) * bs, j * bs:(j + 1) * bs]
                    Ud = Us[j * bs:(j + 1) * bs, j * bs:(j + 1) * bs]
                    assert np.allclose(Lb[blk], Ls[blk] @ np.linalg.inv(Ld), atol=1e-12 * sc)
                    assert np.allclose(Ld @ Ud, Ub[j * bs:(j + 1) * bs, j * bs:(j + 1) * bs], atol=1e-12 * sc)
                else:
                    Ld = Ls[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs]
                    assert np.allclose(Ub[blk], Ld @ Us[blk], atol=1e-12 * sc)


def test_apply_is_the_two_triangular_solves():
    mesh = _mesh((5, 4), 2)
    A = dg.assemble_sipg(mesh)
    il = oilu.ilu0(A.row_ptr, A.col_idx, A.val)
    L, U = oilu.ilu0_dense_factors(il)
    X = dg.random_rhs(A.n, 3, 2)
    Z = oilu.ilu0_apply(il, X)
    # L is unit lower triangular; U is block upper triangular (full diagonal blocks)
    assert np.abs(np.tril(U, -A.bs)).max() == 0
    Zr = np.linalg.solve(U, sla.solve_triangular(L, X, lower=True, unit_diagonal=True))
    assert np.linalg.norm(Z - Zr) <= 1e-12 * np.linalg.norm(Zr)


def test_ilu_iterations_grow_under_h_refinement_while_hss_stays_flat():
    """Sec. 5 (Poisson): with the HSS preconditioner the GMRES iteration count
    does not grow as h is refined; with ILU(0) it does."""
    its_ilu, its_hss = [], []
    for n in (8, 16, 32):
        mesh = _mesh((n, n), 1)
        A = dg.assemble_sipg(mesh)
        Acsr = dg.bsr_to_csr(A)
        b = dg.random_rhs(A.n, 1, 0)[:, 0]
        il = oilu.ilu0(A.row_ptr, A.col_idx, A.val)
        _, i1 = oracle.fgmres(lambda v: Acsr @ v, lambda v: oilu.ilu0_apply(il, v), b, rtol=1e-8, maxit=3000)
        nd = oracle.nd_order(2, mesh.n, 1, A.row_ptr, A.col_idx)
        fac = oracle.factor(Acsr, nd, tol=1e-6, seed=0)
        _, i2 = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8)
        assert i1["converged"] and i2["converged"]
        its_ilu.append(i1["iters"])
        its_hss.append(i2["iters"])
    assert its_ilu[1] >= 1.5 * its_ilu[0] and its_ilu[2] >= 1.5 * its_ilu[1], its_ilu
    assert max(its_hss) - min(its_hss) <= 1 and max(its_hss) < its_ilu[0], its_hss
