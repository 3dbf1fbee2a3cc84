"""The seeded input generator: textbook properties of the SIPG discretisation."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_1508_07798_gb300 import dg_inputs as dg


@pytest.mark.parametrize("dim,n,p", [(2, 4, 1), (2, 5, 2), (2, 3, 3), (3, 3, 1), (3, 3, 2)])
def test_symmetric_and_block_pattern(dim, n, p):
    mesh = dg.Mesh(dim, (n, n, n if dim == 3 else 1), p)
    A = dg.assemble_sipg(mesh)
    D = dg.bsr_to_dense(A)
    assert np.abs(D - D.T).max() <= 1e-13 * np.abs(D).max()
    per_row = np.diff(A.row_ptr)
    assert per_row.max() == 2 * dim + 1
    assert A.val.shape == (A.nnzb, mesh.bs, mesh.bs)
    # each block row holds its diagonal block and sorted neighbours
    for e in range(A.nb):
        cols = A.col_idx[A.row_ptr[e]:A.row_ptr[e + 1]]
        assert np.all(np.diff(cols) > 0) and e in cols


@pytest.mark.parametrize("dim,n,p", [(2, 6, 1), (2, 4, 2), (3, 3, 1)])
def test_poisson_spd(dim, n, p):
    mesh = dg.Mesh(dim, (n, n, n if dim == 3 else 1), p)
    D = dg.bsr_to_dense(dg.assemble_sipg(mesh))
    np.linalg.cholesky(D)


def _l2_error(n, p, dim):
    mesh = dg.Mesh(dim, (n,) * dim + (1,) * (3 - dim), p)
    A = dg.assemble_sipg(mesh)
    lg = dg._legendre_1d(p)
    xg, wg, V = lg["xg"], lg["wg"], lg["V"]
    q = xg.size
    hs = np.array([1.0 / n] * dim)
    cen = dg._elem_centres(mesh)
    qidx = np.stack(np.meshgrid(*([np.arange(q)] * dim), indexing="ij"), axis=-1).reshape(-1, dim)[:, ::-1]
    pts = cen[:, None, :] + 0.5 * hs * xg[qidx][None]
    u = np.prod(np.sin(np.pi * pts), axis=2)
    f = dim * np.pi ** 2 * u
    w = np.prod(wg[qidx], axis=1) * np.prod(hs) / 2 ** dim
    lidx = np.stack(np.meshgrid(*([np.arange(p + 1)] * dim), indexing="ij"), axis=-1).reshape(-1, dim)[:, ::-1]
    phi = np.ones((lidx.shape[0], qidx.shape[0]))
    for k in range(dim):
        phi *= V[lidx[:, k]][:, qidx[:, k]]
    b = ((f * w) @ phi.T).ravel()
    x = spla.spsolve(dg.bsr_to_csr(A).tocsc(), b)
    uh = x.reshape(-1, phi.shape[0]) @ phi
    return math.sqrt(((uh - u) ** 2 * w).sum())


@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_solution_order(p):
    """SIPG converges at order p+1 in L2 for smooth solutions (textbook DG)."""
    e1, e2 = _l2_error(8, p, 2), _l2_error(16, p, 2)
    assert math.log2(e1 / e2) > p + 1 - 0.15


def test_helmholtz_fields_and_kappa():
    mesh, A = dg.helmholtz_2d(16, 2, seed=3)
    c = dg.cosine_field(mesh, 3)
    assert c.min() >= 0.7 - 1e-12 and c.max() <= 1.3 + 1e-12
    assert abs(dg.helmholtz_kappa(64, 2) - 2 * math.pi * 3 * 64 / 10) < 1e-12
    D = dg.bsr_to_dense(A)
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    ev = np.linalg.eigvalsh(D)
    assert ev.min() < 0 < ev.max()           # indefinite


def test_rhs_shapes_and_seeds():
    b1 = dg.random_rhs(100, 3, 7)
    b2 = dg.random_rhs(100, 3, 7)
    assert b1.shape == (100, 3) and b1.flags.f_contiguous and np.array_equal(b1, b2)
    mesh = dg.Mesh(2, (8, 8, 1), 1)
    b = dg.point_source_rhs(mesh, 0)
    assert b.shape == (mesh.ndof, 1) and np.isfinite(b).all() and np.abs(b).max() > 0


def test_diffusion_3d_contrast():
    mesh, A = dg.diffusion_3d(4, 1, seed=0)
    assert A.meta["contrast"] > 10.0
    D = dg.bsr_to_dense(A)
    np.linalg.cholesky(0.5 * (D + D.T))
