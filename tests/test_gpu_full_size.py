"""GPU parity at the full sizes of the workloads, through the C ABI.

* Helmholtz 64 x 64, p = 2 (36,864 dofs, the timed workload, same seeds and
  options): the oracle runs the whole method, so every front, the apply and
  the FGMRES iteration counts are compared.
* Helmholtz 256 x 256, p = 3 (1,048,576 dofs) and 3D diffusion 32^3, p = 1
  (262,144 dofs, 20 right-hand sides): the oracle cannot run the whole
  factorization in seconds, so the checks are (1) the nested dissection,
  bit-exact; (2) sampled boxes whose children were not approximated, where
  S is the exact Schur complement of the box interior (oracle.box_schur) and
  H must stay within the ID tolerance of it; (3) the true FP64 residual of
  every FGMRES solution, computed on the CPU.

At 256 x 256 the FP64 form is also checked on the sampled boxes: S there is
exact, so the oracle's HSS construction of that S (same seed and front id)
must give the GPU's H to 1e-10.

FP32-form tolerance: S of a sampled box comes from eliminating at most a few
dozen interior dofs in FP32 (unit roundoff 6e-8); S32_TOL = 1e-5 relative is
about 20 times the measured worst (4.5e-7).
"""
import numpy as np
import pytest

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
COMPRESSED_TOL = 1e-8
S32_TOL = 1e-5


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _nd_matches(tree, nd):
    ex = tree.export()
    assert ex["level"].tolist() == nd["level"].tolist()
    assert np.array_equal(ex["iset"], nd["iset_flat"])
    assert np.array_equal(ex["bset"], nd["bset_flat"])
    assert np.array_equal(ex["fmap"], nd["fmap_flat"])
    assert np.array_equal(ex["perm"], nd["perm"])


def _true_relres(Acsr, B, X):
    B = B.reshape(B.shape[0], -1)
    X = X.reshape(X.shape[0], -1)
    return (np.linalg.norm(B - Acsr @ X, axis=0) / np.linalg.norm(B, axis=0)).max()


def test_helmholtz_64_p2_timed_workload_matches_oracle():
    """Full size of the timed workload.  Discrete decisions are exact: the
    nested dissection, and per front the largest rank and the final sample
    width.  With compression off (exact LDM^t) every S and the apply agree to
    1e-10.  With compression on, both sides compute the same ranks and
    skeletons, but the map from A to H is ill-conditioned at this size: an
    ID's interpolation matrix T = R11^-1 R12 has cond(R11) up to 1/tol = 1e4
    and the interior blocks reach cond(F_ii) ~ 6e6, so a rounding-level
    difference (u = 1.1e-16, different summation orders) in a child's S can
    grow by 1/tol * cond(F_ii) ~ 6e10 before it reaches an ancestor.  The
    measured worst gap is 1.3e-9 on S and 1.6e-9 on the apply; COMPRESSED_TOL
    = 1e-8 bounds it with a margin of about 6."""
    import torch
    hs = _hss()
    mesh, A = dg.helmholtz_2d(64, 2, 0)
    b = dg.point_source_rhs(mesh, 0)[:, 0]
    Acsr = dg.bsr_to_csr(A)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (64, 64), 2), dA)
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    _nd_matches(tree, nd)
    X = dg.random_rhs(A.n, 2, 11)
    Xd = torch.as_tensor(X, device="cuda")
    # exact mode
    fac0 = oracle.factor(Acsr, nd, compress=False)
    F0 = hs.hss_factor(dA, tree, compress=0, keep_schur=1)
    for bx in range(nd["nbox"]):
        if nd["nb"][bx]:
            assert _rel(F0.export_front(bx)[0], fac0["boxes"][bx]["S"]) <= TOL64, bx
    assert _rel(hs.hss_apply(F0, Xd).cpu().numpy(), oracle.apply(fac0, X)) <= TOL64
    del F0, fac0
    # the method (compression on)
    fac = oracle.factor(Acsr, nd, tol=1e-4, seed=0, rmax=96)
    F = hs.hss_factor(dA, tree, tol=1e-4, seed=0, keep_schur=1)
    logs = {r["box"]: r for r in fac["log"]}
    for bx in range(nd["nbox"]):
        if nd["nb"][bx] == 0:
            continue
        S, H, kmax, r = F.export_front(bx)
        assert _rel(S, fac["boxes"][bx]["S"]) <= COMPRESSED_TOL, bx
        if logs[bx].get("nnodes", 1) > 1:
            assert (kmax, r) == (logs[bx]["kmax"], logs[bx]["r"]), bx
    assert _rel(hs.hss_apply(F, Xd).cpu().numpy(), oracle.apply(fac, X)) <= COMPRESSED_TOL
    xo, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8, restart=30)
    bd = torch.as_tensor(b, device="cuda")
    tol_it = max(1, round(0.1 * info["iters"]))
    # FP64: iterations within 10% of the oracle's.  FP32: the factor's S
    # carries rounding of order cond(F_ii) u_32 in its worst entries, above
    # the ID tolerance in a few fronts, so the ranks there follow rounding
    # order (measured: 6 or 9 of 2,046 fronts differ from FP64, by 1 to 10;
    # 18 or 12 iterations against the oracle's 19).  It must converge to the
    # true residual, be no worse a preconditioner than the oracle's (10%),
    # and keep FP64's ranks on at least 99% of the fronts.
    lg64 = F.export_log()
    for form in ("fp64", "fp32"):
        Ff = F if form == "fp64" else hs.hss_factor(dA, tree, tol=1e-4, seed=0, precision="fp32")
        x, st = hs.fgmres_solve(dA, Ff, bd, rtol=1e-8, restart=30)
        assert st.converged, form
        assert _true_relres(Acsr, b, x.cpu().numpy()) <= 1e-8 * (1 + 1e-6), form
        if form == "fp64":
            assert abs(st.iters - info["iters"]) <= tol_it, (form, st.iters, info["iters"])
        else:
            assert st.iters <= info["iters"] + tol_it, (form, st.iters, info["iters"])
            lg32 = Ff.export_log()
            assert np.array_equal(lg32["box"], lg64["box"])
            assert np.mean(lg32["kmax"] == lg64["kmax"]) >= 0.99


def _single_node_children(nd, bx):
    if nd["is_leaf"][bx]:
        return False
    for c in nd["child"][bx]:
        c = int(c)
        if not nd["is_leaf"][c] or len(oracle.hss_tree_for_front(nd, c)) > 1:
            return False
    return True


def _sample_boxes(nd, count, seed):
    """Up to `count` boxes (seeded order) whose children are leaves with
    single-node HSS trees, so S at the box is exact; boxes with interior dofs
    (which exercise the elimination) first."""
    order = np.random.default_rng(seed).permutation(nd["nbox"])
    with_i, without_i = [], []
    for bx in order:
        bx = int(bx)
        if nd["nb"][bx] == 0 or not _single_node_children(nd, bx):
            continue
        (with_i if nd["ni"][bx] > 0 else without_i).append(bx)
        if len(with_i) >= count:
            break
        if len(with_i) + len(without_i) >= 64 * count:
            break
    return (with_i + without_i)[:count]


LARGE = {
    "helmholtz_256_p3": dict(tol=1e-6),
    "diffusion3d_32_p1": dict(tol=1e-5),
}


@pytest.mark.parametrize("name", sorted(LARGE))
def test_large_workloads_sampled_fronts_and_true_residual(name):
    import torch
    hs = _hss()
    tol = LARGE[name]["tol"]
    if name == "helmholtz_256_p3":
        mesh, A = dg.helmholtz_2d(256, 3, 0)
        B = dg.point_source_rhs(mesh, 0)
        meshd = (2, (256, 256), 3)
    else:
        mesh, A = dg.diffusion_3d(32, 1, 0)
        B = dg.random_rhs(A.n, 20, 0, kind="normal")
        meshd = (3, (32, 32, 32), 1)
    Acsr = dg.bsr_to_csr(A)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order(meshd, dA)
    nd = oracle.nd_order(mesh.dim, mesh.n, mesh.p, A.row_ptr, A.col_idx)
    _nd_matches(tree, nd)
    F = hs.hss_factor(dA, tree, tol=tol, seed=0, precision="fp32", keep_schur=1)
    pick = _sample_boxes(nd, 8, seed=5)
    assert len(pick) == 8
    compressed = 0
    for bx in pick:
        S, H, kmax, r = F.export_front(bx)
        So = oracle.box_schur(Acsr, nd, bx)
        assert _rel(S, So) <= S32_TOL, (bx, _rel(S, So))
        nodes = oracle.hss_tree_for_front(nd, bx)
        depth = max(n_["depth"] for n_ in nodes)
        if len(nodes) > 1:
            compressed += 1
            err = np.linalg.norm(H - So, 2) / np.linalg.norm(So, 2)
            assert err <= 10 * tol * max(depth, 1) + S32_TOL, (bx, err)
    assert compressed > 0
    X, st = hs.fgmres_solve(dA, F, torch.as_tensor(np.asfortranarray(B), device="cuda"), rtol=1e-8,
                            restart=30, maxit=600)
    assert st.converged, (st.iters, st.relres)
    assert _true_relres(Acsr, B, X.cpu().numpy()) <= 1e-8 * (1 + 1e-6)
    if name == "helmholtz_256_p3":
        del F
        F64 = hs.hss_factor(dA, tree, tol=tol, seed=0, keep_schur=1)
        for bx in pick:
            S, H, kmax, r = F64.export_front(bx)
            So = oracle.box_schur(Acsr, nd, bx)
            Ho, rep = oracle.hss_compress(So, oracle.hss_tree_for_front(nd, bx), tol, 0, bx, rmax=96)
            assert _rel(S, So) <= TOL64 and _rel(H, Ho) <= TOL64, bx
