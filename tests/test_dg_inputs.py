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


# --- anisotropic reaction-diffusion (eq. (60)) and the high-contrast density Helmholtz problem

def test_axis_factors_enter_linearly_and_default_is_poisson():
    """Every stiffness, flux, symmetry and penalty term of the faces normal to
    axis k carries K_kk, so A(K) is linear in the axis factors."""
    mesh = dg.Mesh(2, (5, 4, 1), 2)
    Ax = dg.bsr_to_dense(dg.assemble_sipg(mesh, diff_axes=(1.0, 0.0)))
    Ay = dg.bsr_to_dense(dg.assemble_sipg(mesh, diff_axes=(0.0, 1.0)))
    A1 = dg.bsr_to_dense(dg.assemble_sipg(mesh))
    Am = dg.bsr_to_dense(dg.assemble_sipg(mesh, diff_axes=(2.5, 0.01)))
    sc = np.abs(A1).max()
    assert np.abs(Ax + Ay - A1).max() <= 1e-13 * sc
    assert np.abs(2.5 * Ax + 0.01 * Ay - Am).max() <= 1e-13 * sc
    assert np.abs(Ax - Ax.T).max() <= 1e-13 * sc and np.abs(Am - Am.T).max() <= 1e-13 * sc
    with pytest.raises(ValueError):
        dg.assemble_sipg(mesh, diff_axes=(1.0,))


def test_reaction_adds_the_mass_matrix():
    """The orthonormal Legendre basis makes each element's mass matrix
    (|K| / 2^d) I, so +c0 u adds c0 h^2 / 4 to the diagonal in 2D."""
    n = 6
    _, A0 = dg.reaction_diffusion_2d(n, 2, a0=0.1, c0=0.0)
    _, A1 = dg.reaction_diffusion_2d(n, 2, a0=0.1, c0=7.0)
    D = dg.bsr_to_dense(A1) - dg.bsr_to_dense(A0)
    assert np.abs(D - 7.0 / n ** 2 / 4 * np.eye(D.shape[0])).max() <= 1e-12 * np.abs(dg.bsr_to_dense(A0)).max()


def _quad(mesh):
    p, d = mesh.p, 2
    lg = dg._legendre_1d(p)
    q = lg["xg"].size
    hs = np.array([1.0 / mesh.n[0], 1.0 / mesh.n[1]])
    qidx = np.stack(np.meshgrid(*([np.arange(q)] * d), indexing="ij"), axis=-1).reshape(-1, d)[:, ::-1]
    lidx = np.stack(np.meshgrid(*([np.arange(p + 1)] * d), indexing="ij"), axis=-1).reshape(-1, d)[:, ::-1]
    pts = dg._elem_centres(mesh)[:, None, :] + 0.5 * hs * lg["xg"][qidx][None]
    w = np.prod(lg["wg"][qidx], axis=1) * np.prod(hs) / 2 ** d
    phi = np.ones((lidx.shape[0], qidx.shape[0]))
    for k in range(d):
        phi *= lg["V"][lidx[:, k]][:, qidx[:, k]]
    return pts, w, phi


@pytest.mark.parametrize("a0,c0", [(1.0, 0.0), (0.05, 0.0), (0.05, 3.0), (1e-3, 1e3)])
def test_anisotropic_discrete_solution_is_exact_for_a_polynomial(a0, c0):
    """u = x(1-x) y(1-y) lies in the p = 2 space and vanishes on the boundary;
    SIPG is consistent, so the discrete solution of -u_xx - a0 u_yy + c0 u = f
    is u itself (its L2 projection, up to the solve's rounding)."""
    mesh, A = dg.reaction_diffusion_2d(6, 2, a0=a0, c0=c0)
    pts, w, phi = _quad(mesh)
    x, y = pts[..., 0], pts[..., 1]
    u = x * (1 - x) * y * (1 - y)
    f = 2 * y * (1 - y) + a0 * 2 * x * (1 - x) + c0 * u
    b = ((f * w) @ phi.T).ravel()
    # orthonormal basis: the projection coefficients are (u, phi) / (|K| / 4)
    uproj = ((u * w) @ phi.T).ravel() / (1.0 / mesh.nelem / 4.0)
    xs = np.linalg.solve(dg.bsr_to_dense(A), b)
    assert np.abs(xs - uproj).max() <= 1e-9 * np.abs(uproj).max()


def test_enclosure_density_and_operator():
    mesh, A = dg.density_helmholtz_2d(32, 1, rho_ratio=1e3)
    rho = dg.enclosure_density(mesh, 1e3)
    assert set(np.unique(rho)) == {1.0, 1e3}
    g = rho.reshape(32, 32)                       # g[iy, ix]
    # a closed rectangular frame: rows 8..23 and columns 8..23, two elements thick
    frame = np.zeros((32, 32), bool)
    frame[8:24, 8:24] = True
    frame[10:22, 10:22] = False
    assert np.array_equal(g == 1e3, frame)
    assert A.meta["wall_elems"] == frame.sum()
    D = dg.bsr_to_dense(A)
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    # rho_ratio = 1: the plain constant-coefficient Helmholtz operator
    _, A1 = dg.density_helmholtz_2d(32, 1, rho_ratio=1.0)
    ref = dg.assemble_sipg(mesh, kappa=dg.helmholtz_kappa(32, 1))
    assert np.array_equal(A1.val, ref.val) and np.array_equal(A1.col_idx, ref.col_idx)
    # the walls (a = 1e-3) change the blocks of the wall elements and their neighbours only
    dif = np.abs(A.val - ref.val).max(axis=(1, 2)) > 0
    rows = np.repeat(np.arange(A.nb), np.diff(A.row_ptr))
    touched = np.zeros(A.nb, bool)
    touched[rows[dif]] = True
    touched[A.col_idx[dif]] = True
    near = frame.copy()
    near[1:] |= frame[:-1]
    near[:-1] |= frame[1:]
    near[:, 1:] |= frame[:, :-1]
    near[:, :-1] |= frame[:, 1:]
    assert np.array_equal(touched, near.ravel())
