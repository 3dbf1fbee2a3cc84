"""Each step of Algorithm 2 on its own, through the test hooks of the C ABI
(hss_front_eliminate, hss_front_compress), fed the oracle's own input, so a
difference belongs to that step and not to rounding carried in from earlier
levels.

* The timed workload at full size (Helmholtz SIPG p = 2 on 64 x 64 quads,
  ID tolerance 1e-4): at every front the elimination of eq. (32) on the
  oracle's front F gives W = F_ii^-1 F_ib and S = F_bb - F_bi W within 1e-10
  of the oracle's, norm-wise, element-wise and column by column; the stored
  D-block inverse and -F_bi F_ii^-1 are backward stable; and the compression
  (Theorem 1) of the oracle's S gives its H within 1e-10 with the same rank,
  sample width and number of sampling rounds.  Across many levels the full
  factorization drifts further (the map A -> H is ill-conditioned, see
  test_gpu_full_size.py); step by step it does not.
* The blocked Gauss-Jordan sweep of fronts with n >= 2048: on a random front
  with pivoting, and (exact mode) through hss_factor on 3D Poisson 16^3
  p = 1, whose top block has 4,096 rows, every S and the apply against the
  oracle.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg
from parity import rel_col, rel_fro, rel_max

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-10
U64 = np.finfo(np.float64).eps / 2


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


@pytest.fixture(scope="module")
def helm64():
    mesh, A = dg.helmholtz_2d(64, 2, 0)
    Acsr = dg.bsr_to_csr(A)
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    fac = oracle.factor(Acsr, nd, tol=1e-4, seed=0, rmax=96, keep_h=True)
    return mesh, A, nd, fac


def _unpermute(out, perm, ni):
    """The I columns of the transformed front hold F_ii^-1 P^t and
    -F_bi F_ii^-1 P^t: column j belongs to I row perm[j]."""
    inv = np.empty((ni, ni))
    inv[:, perm] = out[:ni, :ni]
    L = np.empty((out.shape[0] - ni, ni))
    L[:, perm] = out[ni:, :ni]
    return inv, L


def _check_elimination(hs, F, ni, ref, tol, precision="fp64", worst=None):
    out, perm, rc = hs.front_eliminate(F, ni, precision=precision)
    assert rc == hs.HSS_OK
    assert sorted(perm.tolist()) == list(range(ni))
    W, S = out[:ni, ni:], out[ni:, ni:]
    errs = dict(W_fro=rel_fro(W, ref["W"]), W_max=rel_max(W, ref["W"]), W_col=rel_col(W, ref["W"]),
                S_fro=rel_fro(S, ref["S"]), S_max=rel_max(S, ref["S"]), S_col=rel_col(S, ref["S"]))
    inv, L = _unpermute(out, perm, ni)
    Fii, Fbi = F[:ni, :ni], F[ni:, :ni]
    # backward errors of the stored blocks (independent of the conditioning)
    errs["inv_bwd"] = np.linalg.norm(Fii @ inv - np.eye(ni)) / (np.linalg.norm(Fii) * np.linalg.norm(inv))
    if L.size:
        errs["L_bwd"] = np.linalg.norm(L @ Fii + Fbi) / (np.linalg.norm(L) * np.linalg.norm(Fii))
    if worst is not None:
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    for k, v in errs.items():
        bound = tol if not k.endswith("_bwd") else (1e-12 if precision == "fp64" else 1e-4)
        assert v <= bound, (k, v, bound)
    return out, perm


def test_elimination_step_at_every_front_of_the_timed_workload(helm64):
    hs = _hss()
    mesh, A, nd, fac = helm64
    worst, nchk = {}, 0
    for b in range(int(nd["nbox"])):
        ni = int(nd["ni"][b])
        if ni == 0:
            continue
        f = fac["boxes"][b]
        _check_elimination(hs, f["F"], ni, f, STEP_TOL, worst=worst)
        nchk += 1
    print(f"\nelimination step, {nchk} fronts, worst: " + ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))
    # the top block A^(0) (eq. (36)) is inverted by the same sweep (every row interior)
    A0 = fac["A0"]
    out, perm, rc = hs.front_eliminate(A0, A0.shape[0])
    assert rc == hs.HSS_OK
    inv, _ = _unpermute(out, perm, A0.shape[0])
    bwd = np.linalg.norm(A0 @ inv - np.eye(A0.shape[0])) / (np.linalg.norm(A0) * np.linalg.norm(inv))
    fwd = rel_fro(inv, sla.lu_solve(fac["top_lu"], np.eye(A0.shape[0])))
    print(f"top block {A0.shape[0]}: backward {bwd:.2e}, against the oracle's inverse {fwd:.2e}")
    assert bwd <= 1e-12 and fwd <= STEP_TOL


def test_compression_step_at_every_front_of_the_timed_workload(helm64):
    hs = _hss()
    mesh, A, nd, fac = helm64
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (64, 64), 2), dA)
    logs = {r["box"]: r for r in fac["log"]}
    worst, ncomp = dict(fro=0.0, max=0.0, col=0.0), 0
    for b in range(int(nd["nbox"])):
        if nd["nb"][b] == 0:
            continue
        f = fac["boxes"][b]
        H, kmax, r, rounds = hs.front_compress(tree, b, f["S"], tol=1e-4, seed=0, rmax=96)
        e = dict(fro=rel_fro(H, f["H"]), max=rel_max(H, f["H"]), col=rel_col(H, f["H"]))
        for k in worst:
            worst[k] = max(worst[k], e[k])
        assert max(e.values()) <= STEP_TOL, (b, e)
        if logs[b].get("nnodes", 1) > 1:
            ncomp += 1
            assert (kmax, r, rounds) == (logs[b]["kmax"], logs[b]["r"], logs[b]["rounds"]), b
    print(f"\ncompression step, {ncomp} compressed fronts, worst: " +
          ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))
    assert ncomp > 100


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_blocked_sweep_on_a_large_random_front(precision):
    """n = 2,400 >= 2,048 takes the blocked sweep (blocks of four 32-column
    panels, the K = 128 update of the columns outside each block); ni = 1,700
    is not a multiple of the block width (a ragged last block).  Random
    normal entries: pivoting is active throughout.  FP64 against the oracle at
    1e-10; FP32 at the bound of its arithmetic, cond(F_ii) * u32 * 64 (the
    sweep's error grows like that of a backward-stable solve)."""
    hs = _hss()
    rng = np.random.default_rng(2400)
    n, ni = 2400, 1700
    F = rng.standard_normal((n, n))
    ref = oracle.eliminate_front(F, ni)
    if precision == "fp64":
        tol = STEP_TOL
    else:
        cond = np.linalg.cond(F[:ni, :ni])
        tol = cond * np.finfo(np.float32).eps / 2 * 64
        print(f"\ncond(F_ii) = {cond:.2e}, FP32 bound {tol:.2e}")
    worst = {}
    _check_elimination(hs, F, ni, ref, tol, precision=precision, worst=worst)
    print(f"{precision}: " + ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_panel_on_a_tall_front(precision):
    """A front with more interior dofs than one CTA's registers hold (ni =
    6,500 > 6,144) takes 32-column panels spread over a thread-block cluster
    (pivot candidates and the pivot row exchanged through distributed shared
    memory); as the panel shortens the cluster shrinks (FP64: 16, 8, 4, 2
    CTAs; FP32: 8, 4, 2) and the last panels run on one CTA.  Random normal
    entries (pivoting throughout) against the oracle's elimination: FP64 at
    1e-10, FP32 at cond(F_ii) u32 64 as for the blocked sweep."""
    hs = _hss()
    rng = np.random.default_rng(6500)
    n, ni = 7000, 6500
    F = rng.standard_normal((n, n))
    ref = oracle.eliminate_front(F, ni)
    if precision == "fp64":
        tol = STEP_TOL
    else:
        cond = np.linalg.cond(F[:ni, :ni])
        tol = cond * np.finfo(np.float32).eps / 2 * 64
        print(f"\ncond(F_ii) = {cond:.2e}, FP32 bound {tol:.2e}")
    hs.profile_reset()
    hs.profile_enable(True)
    worst = {}
    _check_elimination(hs, F, ni, ref, tol, precision=precision, worst=worst)
    hs.profile_enable(False)
    pr = hs.profile_read()
    panel = pr["gj_panel_" + ("f64" if precision == "fp64" else "f32")]
    print(f"{precision}: " + ", ".join(f"{k} {v:.2e}" for k, v in worst.items()) +
          f"; panels {panel[1]} launches, {panel[0]:.1f} ms")


def test_blocked_sweep_exact_mode_3d_poisson():
    """Exact LDM^t (compression off) of 3D Poisson, SIPG p = 1 on 16^3 hexes
    (32,768 dofs): the top block has 4,096 rows and the level-1 and level-2
    fronts exceed 2,048, so the factorization runs the blocked sweep at the
    top of the tree.  Every S and the apply within 1e-10 of the oracle (FP64),
    element-wise; the FP32 factor's apply within the FP32 bound of the
    per-step test, and FGMRES on it converges in a handful of iterations."""
    import torch
    hs = _hss()
    mesh = dg.Mesh(3, (16, 16, 16), 1)
    A = dg.assemble_sipg(mesh)
    Acsr = dg.bsr_to_csr(A)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((3, (16, 16, 16), 1), dA)
    nd = oracle.nd_order(3, mesh.n, 1, A.row_ptr, A.col_idx)
    fac = oracle.factor(Acsr, nd, compress=False)
    big = [b for b in range(int(nd["nbox"])) if nd["ni"][b] + nd["nb"][b] >= 2048]
    assert big and fac["A0"].shape[0] >= 2048
    F = hs.hss_factor(dA, tree, compress=0, keep_schur=1)
    worst = dict(fro=0.0, max=0.0)
    for b in range(int(nd["nbox"])):
        if nd["nb"][b] == 0:
            continue
        S = F.export_front(b)[0]
        ref = fac["boxes"][b]["S"]
        worst["fro"] = max(worst["fro"], rel_fro(S, ref))
        worst["max"] = max(worst["max"], rel_max(S, ref))
    X = dg.random_rhs(A.n, 2, 5)
    Y = hs.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy()
    Yo = oracle.apply(fac, X)
    print(f"\n16^3 exact, {len(big)} fronts >= 2048: S worst {worst}, apply fro {rel_fro(Y, Yo):.2e} "
          f"max {rel_max(Y, Yo):.2e}")
    assert worst["fro"] <= STEP_TOL and worst["max"] <= STEP_TOL
    assert rel_fro(Y, Yo) <= STEP_TOL and rel_max(Y, Yo) <= STEP_TOL
    # FP32 factor of the same problem (blocked sweep in FP32)
    F32 = hs.hss_factor(dA, tree, compress=0, precision="fp32")
    Y32 = hs.hss_apply(F32, torch.as_tensor(X, device="cuda")).cpu().numpy()
    e32 = rel_fro(Y32, Yo)
    b = torch.as_tensor(X[:, 0], device="cuda")
    x, st = hs.fgmres_solve(dA, F32, b, rtol=1e-10, restart=30)
    res = np.linalg.norm(X[:, 0] - Acsr @ x.cpu().numpy()) / np.linalg.norm(X[:, 0])
    print(f"FP32 exact factor: apply against the oracle {e32:.2e}; FGMRES {st.iters} iterations to {res:.2e}")
    assert e32 <= 1e-3
    assert st.converged and res <= 1e-10 and st.iters <= 6
    # the same with the tensor cores: the K = 128 block-end updates of the
    # blocked sweep (16-byte aligned fronts) run on the TMA-fed tcgen05 kernel
    hs.profile_reset()
    hs.profile_enable(True)
    Ftc = hs.hss_factor(dA, tree, compress=0, precision="fp32", tensor_cores=1)
    hs.profile_enable(False)
    cls = hs.profile_read()
    Ytc = hs.hss_apply(Ftc, torch.as_tensor(X, device="cuda")).cpu().numpy()
    etc = rel_fro(Ytc, Yo)
    xt, stt = hs.fgmres_solve(dA, Ftc, b, rtol=1e-10, restart=30)
    rt = np.linalg.norm(X[:, 0] - Acsr @ xt.cpu().numpy()) / np.linalg.norm(X[:, 0])
    tma = [v for k, v in cls.items() if k.startswith("gemm_tma")]
    print(f"FP32 exact factor, tensor cores ({sum(v[1] for v in tma)} TMA launches, "
          f"{sum(v[0] for v in tma):.2f} ms): apply {etc:.2e}; FGMRES {stt.iters} iterations to {rt:.2e}")
    assert tma
    assert etc <= 10 * e32 + 1e-6
    assert stt.converged and rt <= 1e-10 and stt.iters <= st.iters + 1
