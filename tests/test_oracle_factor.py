"""Oracle pins for Algorithm 2, the apply and FGMRES."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg


def _setup(dim, n, p, leaf=64, kind="poisson", seed=0):
    if kind == "poisson":
        mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
        A = dg.assemble_sipg(mesh)
    else:
        mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
        c = dg.cosine_field(mesh, seed)
        A = dg.assemble_sipg(mesh, c_elem=c, kappa=dg.helmholtz_kappa(n[0], p))
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx, leaf_max=leaf)
    return mesh, A, nd, dg.bsr_to_csr(A)


EXACT = [(2, (16, 16), 1, 64, "poisson"), (2, (2, 2), 1, 4, "poisson"), (2, (3, 2), 2, 9, "poisson"),
         (2, (4, 4), 3, 16, "poisson"), (2, (6, 6), 2, 18, "helm"), (3, (2, 2, 2), 1, 8, "poisson"),
         (3, (3, 3, 2), 1, 16, "poisson")]


@pytest.mark.parametrize("dim,n,p,leaf,kind", EXACT)
def test_exact_mode_equals_dense_solve(dim, n, p, leaf, kind):
    """With compression off the LDM^t factorization is exact (Sec. 3/4.1), so
    M^-1 = A^-1: the apply equals a dense LU solve.  Two bars: the normwise
    backward error ||A X - B|| / (||A|| ||X||) <= 1e-15 for every case (the
    dense LU's own is ~1e-17 here), and the forward error against the LU
    solution <= 1e-12, scaled by cond(A) / 1e4 where cond(A) > 1e4 (two
    backward-stable solves of a matrix with cond 5e5, the 6 x 6 Helmholtz
    case, differ by ~cond x eps = 1e-10 at worst; measured 2.3e-12)."""
    mesh, A, nd, Acsr = _setup(dim, n, p, leaf, kind)
    fac = oracle.factor(Acsr, nd, compress=False)
    B = dg.random_rhs(A.n, 3, 1)
    X = oracle.apply(fac, B)
    Ad = Acsr.toarray()
    Xe = np.linalg.solve(Ad, B)
    assert np.linalg.norm(Ad @ X - B) <= 1e-15 * np.linalg.norm(Ad) * np.linalg.norm(X)
    assert np.linalg.norm(X - Xe) <= 1e-12 * np.linalg.norm(Xe) * max(1.0, np.linalg.cond(Ad) / 1e4)


def test_exact_mode_gmres_one_iteration():
    mesh, A, nd, Acsr = _setup(2, (16, 16), 1)
    fac = oracle.factor(Acsr, nd, compress=False)
    b = dg.random_rhs(A.n, 1, 0)[:, 0]
    x, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-10)
    assert info["iters"] == 1 and info["relres"] <= 1e-10


def test_schur_is_inverse_of_trailing_block_of_front_inverse():
    """Sec. 3: the bottom-right block of F^-1 is S^-1."""
    mesh, A, nd, Acsr = _setup(2, (8, 8), 2, 36, "helm")
    fac = oracle.factor(Acsr, nd, tol=1e-6)
    checked = 0
    for b, f in fac["boxes"].items():
        ni = nd["ni"][b]
        if ni == 0 or nd["nb"][b] == 0:
            continue
        Finv = np.linalg.inv(f["F"])
        Sref = np.linalg.inv(Finv[ni:, ni:])
        assert np.linalg.norm(f["S"] - Sref) <= 1e-8 * np.linalg.norm(Sref)
        checked += 1
    assert checked > 5


def test_box_schur_at_leaves_is_inverse_of_trailing_block_of_leaf_inverse():
    """The one-box Schur complement used for sampled checks of large problems,
    at leaves: the trailing block of A(leaf, leaf)^-1 is S^-1 (Sec. 3)."""
    mesh, A, nd, Acsr = _setup(2, (12, 12), 1, 36, "helm")   # 3 x 3-element leaves: one interior element
    leaves = [b for b in range(nd["nbox"]) if nd["is_leaf"][b] and nd["ni"][b] > 0 and nd["nb"][b] > 0]
    assert len(leaves) >= 4
    for b in leaves[:6]:
        S = oracle.box_schur(Acsr, nd, b)
        idx = np.concatenate([nd["iset"][b], nd["bset"][b]])
        Finv = np.linalg.inv(Acsr[idx][:, idx].toarray())
        Sref = np.linalg.inv(Finv[nd["ni"][b]:, nd["ni"][b]:])
        assert np.linalg.norm(S - Sref) <= 1e-10 * np.linalg.norm(Sref)


@pytest.mark.parametrize("dim,n,p,leaf,kind", [(2, (8, 8), 2, 36, "helm"), (3, (4, 4, 4), 1, 64, "poisson")])
def test_box_schur_equals_exact_factor_schur(dim, n, p, leaf, kind):
    """With compression off, Algorithm 2's S at every box equals the Schur
    complement of the box interior taken from A in one step."""
    mesh, A, nd, Acsr = _setup(dim, n, p, leaf, kind)
    fac = oracle.factor(Acsr, nd, compress=False)
    for b in range(nd["nbox"]):
        if nd["nb"][b] == 0:
            continue
        S = oracle.box_schur(Acsr, nd, b)
        ref = fac["boxes"][b]["S"]
        assert np.linalg.norm(S - ref) <= 1e-10 * np.linalg.norm(ref), b


def test_front_assembly_from_children_and_A():
    """eq. (32): a parent front holds H of each child on its diagonal blocks and
    the original couplings A(B^mu, B^nu) across."""
    mesh, A, nd, Acsr = _setup(2, (8, 8), 1, 16)
    fac = oracle.factor(Acsr, nd, compress=False)
    Ad = Acsr.toarray()
    for b in range(nd["nbox"]):
        if nd["is_leaf"][b]:
            continue
        mu, nu = nd["child"][b]
        F = fac["boxes"][b]["F"]
        fm, fn = nd["fmap"][mu], nd["fmap"][nu]
        assert np.array_equal(F[np.ix_(fm, fn)], Ad[np.ix_(nd["bset"][mu], nd["bset"][nu])])
        assert np.allclose(F[np.ix_(fm, fm)], fac["boxes"][mu]["S"], rtol=0, atol=0)


def test_approximate_preconditioner_poisson():
    mesh, A, nd, Acsr = _setup(2, (16, 16), 1)
    fac = oracle.factor(Acsr, nd, tol=1e-6, seed=0)
    b = dg.random_rhs(A.n, 1, 0)[:, 0]
    x, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-10)
    assert info["converged"] and info["iters"] <= 4
    assert np.linalg.norm(b - Acsr @ x) <= 1e-10 * np.linalg.norm(b)
    # compression error of every compressed front stays near the tolerance
    for rec in fac["log"]:
        if rec.get("nnodes", 1) > 1:
            assert rec["kmax"] <= rec["r"] - 10 or rec["r"] >= rec["nb"]


def test_gmres_matches_scipy_unpreconditioned():
    mesh, A, nd, Acsr = _setup(2, (6, 6), 1)
    b = dg.random_rhs(A.n, 1, 2)[:, 0]
    x, info = oracle.fgmres(lambda v: Acsr @ v, None, b, restart=20, rtol=1e-9, maxit=20)
    ref = []
    spla.gmres(Acsr, b, restart=20, maxiter=1, rtol=1e-30, callback=lambda r: ref.append(r),
               callback_type="pr_norm")
    ref = np.array(ref)
    ours = np.array(info["hist"][: ref.size])
    assert ref.size >= 10
    assert np.allclose(ours, ref, rtol=1e-7, atol=1e-14)


def test_gmres_restart_and_nonconvergence():
    mesh, A, nd, Acsr = _setup(2, (8, 8), 1)
    b = dg.random_rhs(A.n, 1, 3)[:, 0]
    x, info = oracle.fgmres(lambda v: Acsr @ v, None, b, restart=5, rtol=1e-8, maxit=2000)
    assert info["converged"]
    assert np.linalg.norm(b - Acsr @ x) <= 1e-8 * np.linalg.norm(b)
    x2, info2 = oracle.fgmres(lambda v: Acsr @ v, None, b, restart=5, rtol=1e-12, maxit=3)
    assert not info2["converged"] and info2["iters"] == 3


# --- sample-width cap policies (Theorem 1 needs k + p samples; Sec. 5 fixes the width l)

def _capped_runs(r=16):
    mesh, A, nd, Acsr = _setup(2, (16, 16), 1, kind="helm")
    kw = dict(tol=1e-12, seed=5, r0=r, rmax=r, keep_h=True)
    return nd, oracle.factor(Acsr, nd, cap="keep", **kw), oracle.factor(Acsr, nd, cap="accept", **kw)


def test_cap_policies_differ_only_on_capped_fronts():
    nd, fk, fa = _capped_runs()
    capped = {r["box"] for r in fk["log"] if r.get("capped")}
    assert capped and capped == {r["box"] for r in fa["log"] if r.get("capped")}
    for b in fk["boxes"]:
        Hk, Ha, S = fk["boxes"][b]["H"], fa["boxes"][b]["H"], fk["boxes"][b]["S"]
        if b in capped:
            assert np.array_equal(Hk, S) and not np.array_equal(Ha, S)
        else:
            assert np.array_equal(Hk, Ha)
    with pytest.raises(ValueError):
        oracle.factor(dg.bsr_to_csr(dg.poisson_2d(16, 1)[1]), nd, cap="drop")


def test_accepted_approximant_is_hss_with_ranks_at_most_r():
    """Under the accept policy a capped front's H keeps the nested-basis
    structure: for every HSS node a, the off-diagonal block row H(R_a, ~R_a)
    lies in the span of U^tall_a, so its rank is at most the sample width."""
    nd, fk, fa = _capped_runs(r=8)
    checked = 0
    for rec in fa["log"]:
        if not rec.get("capped"):
            continue
        H, S = fa["boxes"][rec["box"]]["H"], fa["boxes"][rec["box"]]["S"]
        nodes = rec["rep"]["nodes"]
        for t, nd_ in enumerate(nodes[:-1]):
            R = np.arange(nd_["lo"], nd_["hi"])
            C_ = np.setdiff1d(np.arange(H.shape[0]), R)
            sv = np.linalg.svd(H[np.ix_(R, C_)], compute_uv=False)
            assert (sv > 1e-11 * sv[0]).sum() <= rec["r"], (rec["box"], t)
            full = np.linalg.svd(S[np.ix_(R, C_)], compute_uv=False)
            checked += (full > 1e-11 * full[0]).sum() > rec["r"]
    assert checked > 0          # somewhere S itself needed more than r


def test_partition_scheme_matters_for_anisotropic_diffusion():
    """Sec. 5, eq. (60) with the printed anisotropy a0 = 1e-6 (Fig. 10) and a
    fixed sample width l = 16, at the printed c0 = 1e-4, 1, 1e2, 1e3: vertical
    slabs (cuts across the strong x coupling; the coupling between a slab's
    left and right boundaries is one full-rank x chain per row) fail while
    horizontal slabs converge.  The scheme stops mattering once reaction
    dominates at the element scale (c0 h^2 >> 1; c0 = 1e6 at h = 1/16, beyond
    the printed values)."""
    its = {}
    for c0 in (1e-4, 1.0, 1e2, 1e3, 1e6):
        mesh, A = dg.reaction_diffusion_2d(16, 1, a0=1e-6, c0=c0)
        Acsr = dg.bsr_to_csr(A)
        b = dg.random_rhs(A.n, 1, 0)[:, 0]
        for sc in ("hslab", "vslab"):
            nd = oracle.nd_order(2, mesh.n, 1, A.row_ptr, A.col_idx, scheme=sc)
            fac = oracle.factor(Acsr, nd, tol=1e-12, seed=0, r0=16, rmax=16, cap="accept")
            _, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8,
                                    restart=30, maxit=120)
            its[c0, sc] = info["iters"] if info["converged"] else None
    for c0 in (1e-4, 1.0, 1e2, 1e3):
        assert its[c0, "hslab"] is not None and its[c0, "hslab"] <= 5 and its[c0, "vslab"] is None, its
    assert its[1e6, "vslab"] is not None and its[1e6, "vslab"] <= 30, its


# --- residual probe of accepted approximants (fallback check of the learned widths)

def test_probe_leaves_healthy_runs_unchanged():
    """With oversampling 10 every front passes the probe: the approximants are
    those of the run without it, and each probe ratio is within its threshold."""
    mesh, A, nd, Acsr = _setup(2, (16, 16), 2, kind="helm")
    f0 = oracle.factor(Acsr, nd, tol=1e-6, seed=1, rmax=96, keep_h=True)
    f1 = oracle.factor(Acsr, nd, tol=1e-6, seed=1, rmax=96, keep_h=True, probe=4)
    for b in f0["boxes"]:
        assert np.array_equal(f0["boxes"][b]["H"], f1["boxes"][b]["H"])
    recs = [r for r in f1["log"] if r.get("nnodes", 1) > 1]
    assert recs and all(r["probe_regrown"] == 0 for r in recs)
    for r in recs:
        assert r["probe_rel"] <= oracle.probe_threshold(1e-6, r["rep"]["nodes"])


def test_probe_catches_undersampled_fronts():
    """Without oversampling (p = 0) the rank test never asks for more samples;
    the probe does, and the regrown fronts pass it at their final width."""
    mesh, A, nd, Acsr = _setup(2, (16, 16), 2, kind="helm")
    kw = dict(tol=1e-6, seed=1, r0=8, rmax=96, oversample=0)
    f0 = oracle.factor(Acsr, nd, **kw)
    f1 = oracle.factor(Acsr, nd, probe=4, **kw)
    recs = [r for r in f1["log"] if r.get("nnodes", 1) > 1]
    assert sum(r["probe_regrown"] for r in recs) > 0
    assert all(r["rounds"] == 1 for r in f0["log"] if r.get("nnodes", 1) > 1)
    for r in recs:
        if not r["capped"]:
            assert r["probe_rel"] <= oracle.probe_threshold(1e-6, r["rep"]["nodes"])
    b = dg.random_rhs(A.n, 1, 0)[:, 0]
    its = []
    for fac in (f0, f1):
        _, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8, maxit=300)
        its.append(info["iters"] if info["converged"] else 10 ** 6)
    assert its[1] < its[0], its


def test_eliminate_front_is_the_schur_complement_definition():
    """oracle.eliminate_front on a random front (partial pivoting needed: no
    diagonal dominance): S equals the inverse of the trailing block of F^-1
    (the Schur-complement identity, independent of how S is computed), W
    solves F_ii W = F_ib, and with no interior dofs S is F itself."""
    rng = np.random.default_rng(12)
    n, ni = 300, 170
    F = rng.standard_normal((n, n))
    el = oracle.eliminate_front(F, ni)
    S_id = np.linalg.inv(np.linalg.inv(F)[ni:, ni:])
    assert np.linalg.norm(el["S"] - S_id) / np.linalg.norm(S_id) <= 1e-10
    res = np.linalg.norm(F[:ni, :ni] @ el["W"] - F[:ni, ni:])
    assert res <= 1e-13 * np.linalg.norm(F[:ni, :ni]) * np.linalg.norm(el["W"])   # backward stable
    e0 = oracle.eliminate_front(F[:40, :40], 0)
    assert e0["lu"] is None and np.array_equal(e0["S"], F[:40, :40])
