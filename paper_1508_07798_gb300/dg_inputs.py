"""Seeded synthetic test inputs: SIPG discontinuous-Galerkin system matrices.

This module produces the *inputs* of the method (a sparse matrix A in block
CSR form, its structured element grid, and right-hand sides).  It holds none
of the method's arithmetic: no ordering, elimination, compression or Krylov
step lives here.  It is shared, as data, by the CPU oracle, the GPU tests and
the benchmark.

Discretisation (paper Sec. 5 uses interior-penalty DG on the unit square; the
operators below are the ones of Sec. 5, on uniform quadrilateral/hexahedral
grids with an orthonormal tensor-Legendre basis per element):

    -div(a K grad u) - kappa^2 c(x) u + r u = f  in (0,1)^d,   u = 0 on the boundary,

K = diag(s_x, s_y[, s_z]) a constant axis-aligned diffusion tensor (identity
unless given; the anisotropic reaction-diffusion problem, eq. (60)), symmetric
interior penalty with penalty sigma_e = 10 p^2 / h * max(a-, a+) * (n.K.n),
(p+2)-point Gauss rules, element-wise constant a and c.  Element e has the
lexicographic index e = ix + nx*(iy + ny*iz); its local dof l = a + (p+1)*b
(+ (p+1)^2 * c in 3D) belongs to the basis function L_a(xi) L_b(eta) [L_c(zeta)];
the global dof is e*bs + l with bs = (p+1)^d.

Block CSR layout: one block row per element, block columns sorted ascending,
each block a dense bs x bs row-major array (row = test function, column = trial
function).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "BSR", "assemble_sipg", "poisson_2d", "helmholtz_2d", "diffusion_3d",
    "reaction_diffusion_2d", "density_helmholtz_2d", "enclosure_density", "helmholtz_kappa",
    "bsr_to_csr", "bsr_to_dense", "random_rhs", "point_source_rhs",
    "splitmix64",
]


@dataclass
class Mesh:
    """Uniform element grid on the unit square/cube."""
    dim: int
    n: tuple          # elements per axis, length 3 (unused axes = 1)
    p: int

    @property
    def bs(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def nelem(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    @property
    def ndof(self) -> int:
        return self.nelem * self.bs


@dataclass
class BSR:
    """Square block-sparse matrix, bs x bs row-major blocks, int32 indices."""
    nb: int
    bs: int
    row_ptr: np.ndarray   # int32 [nb+1]
    col_idx: np.ndarray   # int32 [nnzb]
    val: np.ndarray       # float64 [nnzb, bs, bs]
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nb * self.bs

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])


# --------------------------------------------------------------------------
# counter-based generator (published SplitMix64 finaliser, Steele/Lea/Flood
# 2014 as popularised by Vigna): used only to derive reproducible seeds here.
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


# --------------------------------------------------------------------------
# 1D orthonormal Legendre data on [-1, 1]
# --------------------------------------------------------------------------
def _legendre_1d(p: int):
    q = p + 2
    xg, wg = np.polynomial.legendre.leggauss(q)
    V = np.zeros((p + 1, q))        # L_a(x_q)
    D = np.zeros((p + 1, q))        # L_a'(x_q)
    vm = np.zeros(p + 1)            # L_a(-1)
    vp = np.zeros(p + 1)            # L_a(+1)
    dm = np.zeros(p + 1)            # L_a'(-1)
    dp = np.zeros(p + 1)            # L_a'(+1)
    for a in range(p + 1):
        c = np.zeros(a + 1)
        c[a] = math.sqrt((2 * a + 1) / 2.0)
        dc = np.polynomial.legendre.legder(c) if a > 0 else np.zeros(1)
        V[a] = np.polynomial.legendre.legval(xg, c)
        D[a] = np.polynomial.legendre.legval(xg, dc)
        vm[a] = np.polynomial.legendre.legval(-1.0, c)
        vp[a] = np.polynomial.legendre.legval(1.0, c)
        dm[a] = np.polynomial.legendre.legval(-1.0, dc)
        dp[a] = np.polynomial.legendre.legval(1.0, dc)
    M1 = (V * wg) @ V.T             # = I up to rounding
    K1 = (D * wg) @ D.T
    return dict(xg=xg, wg=wg, V=V, D=D, vm=vm, vp=vp, dm=dm, dp=dp, M1=M1, K1=K1)


def _kron_axes(mats):
    """Kronecker product with axis 0 fastest: mats[0] acts on the x index."""
    out = np.ones((1, 1))
    for m in mats:               # x first, then y, then z
        out = np.kron(m, out)
    return out


def assemble_sipg(mesh: Mesh, a_elem=None, c_elem=None, kappa: float = 0.0,
                  penalty: float = 10.0, diff_axes=None, reaction: float = 0.0) -> BSR:
    """Assemble the SIPG matrix of -div(a K grad u) - kappa^2 c u + reaction u on (0,1)^d.

    a_elem, c_elem: per-element constants (default 1).  diff_axes: the
    diagonal of K, one factor per axis (default all 1).  K scales the axis-k
    stiffness and every term of the faces normal to axis k (flux, symmetry
    and penalty, since n.K.n = K_kk there), so the matrix is linear in K when
    kappa = reaction = 0.  Dirichlet u=0 on all boundary faces, imposed weakly
    by one-sided fluxes.
    """
    d, p = mesh.dim, mesh.p
    n = tuple(int(v) for v in mesh.n[:d])
    ne = mesh.nelem
    bs = mesh.bs
    h = [1.0 / n[k] for k in range(d)]
    lg = _legendre_1d(p)
    I1 = np.eye(p + 1)
    M1, K1 = lg["M1"], lg["K1"]
    a_elem = np.ones(ne) if a_elem is None else np.asarray(a_elem, dtype=np.float64)
    c_elem = np.ones(ne) if c_elem is None else np.asarray(c_elem, dtype=np.float64)
    kdiag = np.ones(d) if diff_axes is None else np.asarray(diff_axes, dtype=np.float64)
    if kdiag.shape != (d,) or (kdiag < 0).any():
        raise ValueError("diff_axes: one non-negative factor per axis")
    vol = float(np.prod(h))

    # volume: stiffness per axis and mass
    stiff = np.zeros((bs, bs))
    for k in range(d):
        mats = [K1 if j == k else M1 for j in range(d)]
        scale = kdiag[k] * vol * (2.0 / h[k]) ** 2 / 2.0 ** d
        stiff += scale * _kron_axes(mats)
    mass = (vol / 2.0 ** d) * _kron_axes([M1] * d)

    diag = (a_elem[:, None, None] * stiff[None] - (kappa ** 2) * c_elem[:, None, None] * mass[None]
            + reaction * mass[None])

    idx = np.arange(ne).reshape(tuple(reversed(n)))  # idx[iz][iy][ix]

    sides = {  # trace value, derivative value, jump sign for the lower (-) and upper (+) element
        "lo": (lg["vp"], lg["dp"], +1.0),   # element below/left of the face: its xi=+1 side
        "hi": (lg["vm"], lg["dm"], -1.0),   # element above/right: its xi=-1 side
    }

    # off-diagonal blocks collected as (row element, column element, block)
    orow, ocol, oblk = [], [], []
    idx3 = idx.reshape((1,) * (3 - d) + idx.shape)
    for k in range(d):
        fscale = kdiag[k] * vol / h[k] / 2.0 ** (d - 1)   # K_kk * face measure / reference face measure
        g = 2.0 / h[k]
        ax = 2 - k                              # axis k inside idx3 (z, y, x order)

        def lift(f1):
            """Tensor the 1D face factor along axis k with identities elsewhere."""
            mats = [I1] * d
            mats[k] = f1
            return fscale * _kron_axes(mats)

        # interior faces normal to axis k: element lo (its xi_k=+1 side) and hi
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        e_lo = idx3[tuple(sl_lo)].ravel()
        e_hi = idx3[tuple(sl_hi)].ravel()
        if e_lo.size:
            alo, ahi = a_elem[e_lo], a_elem[e_hi]
            sig = penalty * p * p / h[k] * np.maximum(alo, ahi)

            def blocks(s, t, a_s, a_t):
                vs, ds, js = sides[s]
                vt, dt, jt = sides[t]
                P1 = lift(-0.5 * g * js * np.outer(vs, dt))
                P2 = lift(-0.5 * g * jt * np.outer(ds, vt))
                P3 = lift(js * jt * np.outer(vs, vt))
                return (a_t[:, None, None] * P1[None] + a_s[:, None, None] * P2[None]
                        + sig[:, None, None] * P3[None])

            np.add.at(diag, e_lo, blocks("lo", "lo", alo, alo))
            np.add.at(diag, e_hi, blocks("hi", "hi", ahi, ahi))
            orow += [e_lo, e_hi]
            ocol += [e_hi, e_lo]
            oblk += [blocks("lo", "hi", alo, ahi), blocks("hi", "lo", ahi, alo)]
        # boundary faces normal to axis k: -a d_n u v - a d_n v u + sig u v,
        # d_n = js * d/dx_k.  Low wall: element's xi=-1 side ("hi" role, outward
        # normal -e_k); high wall: xi=+1 side ("lo" role, outward normal +e_k).
        for s, pos in (("hi", 0), ("lo", -1)):
            sl = [slice(None)] * 3
            sl[ax] = pos
            eb = idx3[tuple(sl)].ravel()
            ab = a_elem[eb]
            sig = penalty * p * p / h[k] * ab
            vs, ds, js = sides[s]
            Q1 = lift(-g * js * (np.outer(vs, ds) + np.outer(ds, vs)))
            Q3 = lift(np.outer(vs, vs))
            np.add.at(diag, eb, ab[:, None, None] * Q1[None] + sig[:, None, None] * Q3[None])

    erow = np.concatenate(orow + [np.arange(ne)])
    ecol = np.concatenate(ocol + [np.arange(ne)])
    eblk = np.concatenate(oblk + [diag]) if oblk else diag
    order = np.lexsort((ecol, erow))
    erow, ecol, eblk = erow[order], ecol[order], eblk[order]
    row_ptr = np.zeros(ne + 1, dtype=np.int32)
    np.add.at(row_ptr, erow + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return BSR(nb=ne, bs=bs, row_ptr=row_ptr, col_idx=ecol.astype(np.int32),
               val=np.ascontiguousarray(eblk, dtype=np.float64),
               meta=dict(dim=d, n=n, p=p, kappa=kappa, diff_axes=tuple(float(v) for v in kdiag),
                         reaction=reaction))


# --------------------------------------------------------------------------
# problem families (paper Sec. 5 operators; shapes of the benchmark configs)
# --------------------------------------------------------------------------
def _elem_centres(mesh: Mesh) -> np.ndarray:
    d = mesh.dim
    n = mesh.n[:d]
    grids = np.meshgrid(*[(np.arange(n[k]) + 0.5) / n[k] for k in reversed(range(d))], indexing="ij")
    # grids[j] varies along reversed axis j; reorder to (x, y, z)
    cen = np.stack([g.ravel() for g in reversed(grids)], axis=1)
    return cen


def helmholtz_kappa(n: int, p: int, dofs_per_wavelength: float = 10.0) -> float:
    """Wave number with a fixed number of dofs per wavelength: (p+1)/h dofs per
    unit length, so kappa = 2 pi (p+1) n / dofs_per_wavelength (the paper keeps
    the dispersion error constant under h/p refinement, Sec. 5)."""
    return 2.0 * math.pi * (p + 1) * n / dofs_per_wavelength


def cosine_field(mesh: Mesh, seed: int, nterms: int = 8, amp: float = 0.3) -> np.ndarray:
    """c(x) = 1 + amp * mean_j cos(2 pi k_j.x + phi_j), k_j in {1..4}^d, evaluated at
    element centres (piecewise constant, as the paper's element-wise density)."""
    rng = np.random.default_rng(seed)
    kv = rng.integers(1, 5, size=(nterms, mesh.dim))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=nterms)
    x = _elem_centres(mesh)
    s = np.cos(2.0 * math.pi * x @ kv.T + ph[None, :]).mean(axis=1)
    return 1.0 + amp * s


def gaussian_log_field(mesh: Mesh, seed: int, variance: float = 2.0, m: int = 64,
                       corr: float = 0.1) -> np.ndarray:
    """g(x) = sqrt(variance) sqrt(2/m) sum_m cos(w_m.x + t_m) (random Fourier features of a
    smooth Gaussian field), a = exp(g) per element centre."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 2.0 * math.pi / corr, size=(m, mesh.dim))
    t = rng.uniform(0.0, 2.0 * math.pi, size=m)
    x = _elem_centres(mesh)
    g = math.sqrt(variance) * math.sqrt(2.0 / m) * np.cos(x @ w.T + t[None, :]).sum(axis=1)
    return np.exp(g)


def poisson_2d(n: int, p: int) -> tuple:
    mesh = Mesh(2, (n, n, 1), p)
    return mesh, assemble_sipg(mesh)


def helmholtz_2d(n: int, p: int, seed: int, kappa: float | None = None) -> tuple:
    mesh = Mesh(2, (n, n, 1), p)
    kap = helmholtz_kappa(n, p) if kappa is None else kappa
    c = cosine_field(mesh, seed)
    A = assemble_sipg(mesh, c_elem=c, kappa=kap)
    A.meta.update(c_mean=float(c.mean()), c_var=float(c.var()))
    return mesh, A


def diffusion_3d(n: int, p: int, seed: int) -> tuple:
    mesh = Mesh(3, (n, n, n), p)
    a = gaussian_log_field(mesh, seed)
    A = assemble_sipg(mesh, a_elem=a)
    A.meta.update(contrast=float(a.max() / a.min()))
    return mesh, A


def reaction_diffusion_2d(n: int, p: int, a0: float, c0: float) -> tuple:
    """Constant-coefficient anisotropic reaction-diffusion, eq. (60) divided by
    a_11: -u_xx - a0 u_yy + c0 u = f0 (a0 = a_22/a_11, c0 = c/a_11), with
    a0 << 1 making the x direction the strongly coupled one (Sec. 5)."""
    mesh = Mesh(2, (n, n, 1), p)
    A = assemble_sipg(mesh, diff_axes=(1.0, a0), reaction=c0)
    A.meta.update(a0=a0, c0=c0)
    return mesh, A


def enclosure_density(mesh: Mesh, rho_d: float, rho_0: float = 1.0, box=(0.25, 0.75, 0.25, 0.75),
                      wall: float = 1.0 / 16) -> np.ndarray:
    """Element-wise density of the high-contrast Helmholtz problem (Sec. 5): a
    rectangular enclosure D -- the walls, of thickness `wall`, of the
    rectangle [x0, x1] x [y0, y1] given by `box` -- has density rho_d, the
    rest of the unit square rho_0.  An element belongs to D when its centre
    does (at least one element across each wall)."""
    x0, x1, y0, y1 = box
    cen = _elem_centres(mesh)
    x, y = cen[:, 0], cen[:, 1]
    hx, hy = 1.0 / mesh.n[0], 1.0 / mesh.n[1]
    tx, ty = max(wall, hx), max(wall, hy)
    inside_outer = (x > x0) & (x < x1) & (y > y0) & (y < y1)
    inside_inner = (x > x0 + tx) & (x < x1 - tx) & (y > y0 + ty) & (y < y1 - ty)
    return np.where(inside_outer & ~inside_inner, rho_d, rho_0)


def density_helmholtz_2d(n: int, p: int, rho_ratio: float = 1e3, kappa: float | None = None) -> tuple:
    """-div(rho^-1 grad u) - kappa^2 u = f with the piecewise-constant density
    of `enclosure_density` (rho_0 = 1, rho_d = rho_ratio); kappa defaults to
    the same 10 dofs per wavelength as `helmholtz_2d` (with respect to rho_0)."""
    mesh = Mesh(2, (n, n, 1), p)
    kap = helmholtz_kappa(n, p) if kappa is None else kappa
    rho = enclosure_density(mesh, rho_ratio)
    A = assemble_sipg(mesh, a_elem=1.0 / rho, kappa=kap)
    A.meta.update(rho_ratio=rho_ratio, wall_elems=int((rho != 1.0).sum()))
    return mesh, A


def rank_training_problems(n: int = 64, ps=(1, 2, 3), seeds=range(100, 116)) -> list:
    """Helmholtz problems whose adaptive factorizations give the training ranks
    of the learned-width form: (mesh descriptor, matrix, c per element,
    kappa * h) for every p in ps and seed in seeds (the default: 64 x 64
    quads, p = 1, 2, 3, seeds 100..115)."""
    out = []
    for p in ps:
        for sd in seeds:
            mesh, A = helmholtz_2d(n, p, sd)
            out.append(((2, (n, n), p), A, cosine_field(mesh, sd), helmholtz_kappa(n, p) / n))
    return out


def diffusion_training_problems(n: int = 16, p: int = 1, seeds=range(100, 116)) -> list:
    """3D diffusion problems (a = exp(g) per `diffusion_3d`) whose adaptive
    factorizations give training ranks for the 3D learned-width form: (mesh
    descriptor, matrix, log a per element, kappa * h = 0) per seed."""
    out = []
    for sd in seeds:
        mesh, A = diffusion_3d(n, p, sd)
        out.append(((3, (n, n, n), p), A, np.log(gaussian_log_field(mesh, sd)), 0.0))
    return out


def random_rhs(ndof: int, nrhs: int, seed: int, kind: str = "uniform") -> np.ndarray:
    """Column-major (ndof x nrhs) right-hand sides: U(-1,1) or N(0,1) per dof."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        b = rng.uniform(-1.0, 1.0, size=(nrhs, ndof))
    else:
        b = rng.standard_normal(size=(nrhs, ndof))
    return np.asfortranarray(b.T)


def point_source_rhs(mesh: Mesh, seed: int) -> np.ndarray:
    """b_i = integral of f phi_i with f a Gaussian of width 2h at a random x0 in (0.25,0.75)^d."""
    rng = np.random.default_rng(seed)
    d, p = mesh.dim, mesh.p
    n = mesh.n[:d]
    h = 1.0 / n[0]
    x0 = rng.uniform(0.25, 0.75, size=d)
    lg = _legendre_1d(p)
    xg, wg, V = lg["xg"], lg["wg"], lg["V"]
    q = xg.size
    cen = _elem_centres(mesh)                       # (ne, d)
    hs = np.array([1.0 / n[k] for k in range(d)])
    # quadrature points per element: tensor grid, x fastest
    qidx = np.stack(np.meshgrid(*([np.arange(q)] * d), indexing="ij"), axis=-1).reshape(-1, d)[:, ::-1]
    pts = cen[:, None, :] + 0.5 * hs[None, None, :] * xg[qidx][None, :, :]
    f = np.exp(-((pts - x0) ** 2).sum(axis=2) / (2.0 * (2.0 * h) ** 2))   # (ne, q^d)
    w = np.prod(wg[qidx], axis=1) * np.prod(hs) / 2.0 ** d                # (q^d,)
    lidx = np.stack(np.meshgrid(*([np.arange(p + 1)] * d), indexing="ij"), axis=-1).reshape(-1, d)[:, ::-1]
    phi = np.ones((lidx.shape[0], qidx.shape[0]))
    for k in range(d):
        phi *= V[lidx[:, k]][:, qidx[:, k]]
    b = (f * w[None, :]) @ phi.T                                           # (ne, bs)
    return np.asfortranarray(b.reshape(-1, 1))


def batched_instances(count: int, master_seed: int = 0, n_range=(16, 64), p_set=(1, 2, 3),
                      ops=("poisson", "helmholtz")):
    """Independent problems of the batched workload: per instance i the seed
    splitmix64(master_seed + i) draws the mesh size n ~ U{n_range}, the degree
    p from p_set and the operator (Bernoulli 1/2 over ops); Helmholtz takes
    10 dofs per wavelength and c(x) per cosine_field, Poisson a = 1.  Returns
    a list of dicts (mesh, A, kind, seed)."""
    out = []
    for i in range(count):
        sd = splitmix64(master_seed + i)
        n = n_range[0] + int(sd % (n_range[1] - n_range[0] + 1))
        p = p_set[int((sd >> 16) % len(p_set))]
        kind = ops[int((sd >> 32) % len(ops))]
        seed = int((sd >> 40) & 0xFFFF)
        if kind == "poisson":
            mesh, A = poisson_2d(n, p)
        else:
            mesh, A = helmholtz_2d(n, p, seed)
        out.append(dict(mesh=mesh, A=A, kind=kind, seed=seed))
    return out


def bsr_to_csr(A: BSR):
    """scipy CSR copy of the block matrix (row-major blocks)."""
    import scipy.sparse as sp
    M = sp.bsr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.n, A.n))
    return M.tocsr()


def bsr_to_dense(A: BSR) -> np.ndarray:
    return bsr_to_csr(A).toarray()
