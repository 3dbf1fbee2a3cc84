"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars: nested-dissection sets, maps and permutation bit-exact; Schur
complements, HSS approximants and the preconditioner apply within 1e-10
relative in FP64; FGMRES reaches the same relative residual with iteration
counts within +-10% (at least +-1).
"""
import numpy as np
import pytest

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def _setup(kind, n, p, dim=2, seed=0, leaf=64):
    if kind == "poisson":
        mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
        A = dg.assemble_sipg(mesh)
    elif kind == "helm":
        mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
        c = dg.cosine_field(mesh, seed)
        A = dg.assemble_sipg(mesh, c_elem=c, kappa=dg.helmholtz_kappa(n[0], p))
    else:
        mesh = dg.Mesh(3, tuple(n), p)
        A = dg.assemble_sipg(mesh, a_elem=dg.gaussian_log_field(mesh, seed))
    return mesh, A


ND_CASES = [("poisson", (16, 16), 1, 2, 64), ("poisson", (2, 1), 1, 2, 4), ("poisson", (7, 5), 2, 2, 18),
            ("helm", (6, 6), 3, 2, 16), ("poisson", (3, 3, 2), 1, 3, 16), ("poisson", (4, 4, 4), 1, 3, 64),
            ("poisson", (5, 4), 1, 2, 1000), ("helm", (64, 64), 2, 2, 64)]


@pytest.mark.parametrize("scheme", ["box", "hslab", "vslab"])
@pytest.mark.parametrize("kind,n,p,dim,leaf", ND_CASES)
def test_nd_bit_exact(kind, n, p, dim, leaf, scheme):
    if scheme != "box" and n[0] > 16:
        pytest.skip("slab schemes checked on the small meshes")
    hs = _hss()
    mesh, A = _setup(kind, n, p, dim)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((dim, tuple(n), p), dA, leaf_max=leaf, scheme=scheme)
    ex = tree.export()
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx, leaf_max=leaf, scheme=scheme)
    assert ex["level"].tolist() == nd["level"].tolist()
    assert ex["parent"].tolist() == nd["parent"].tolist()
    assert ex["child0"].tolist() == nd["child"][:, 0].tolist()
    assert ex["child1"].tolist() == nd["child"][:, 1].tolist()
    assert np.array_equal(ex["lohi"][:, :3], nd["lo"]) and np.array_equal(ex["lohi"][:, 3:], nd["hi"])
    assert ex["ni"].tolist() == nd["ni"].tolist() and ex["nb"].tolist() == nd["nb"].tolist()
    assert np.array_equal(ex["iset"], nd["iset_flat"])
    assert np.array_equal(ex["bset"], nd["bset_flat"])
    assert np.array_equal(ex["fmap"], nd["fmap_flat"])
    assert np.array_equal(ex["perm"], nd["perm"])


def test_spmv_matches_scipy():
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (16, 16), 2)
    dA = hs.DeviceBSR.from_host(A)
    X = dg.random_rhs(A.n, 3, 5)
    Y = hs.hss_spmv(dA, torch.as_tensor(X, device="cuda")).cpu().numpy()
    ref = dg.bsr_to_csr(A) @ X
    assert np.linalg.norm(Y - ref) <= 1e-14 * np.linalg.norm(ref)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


EXACT = [("poisson", (16, 16), 1, 2, 64), ("helm", (12, 12), 2, 2, 36), ("poisson", (2, 1), 1, 2, 4),
         ("poisson", (3, 3, 3), 1, 3, 16), ("helm", (9, 7), 3, 2, 32)]


@pytest.mark.parametrize("kind,n,p,dim,leaf", EXACT)
def test_exact_mode_apply_equals_oracle_and_dense_solve(kind, n, p, dim, leaf):
    import torch
    hs = _hss()
    mesh, A = _setup(kind, n, p, dim)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((dim, tuple(n), p), dA, leaf_max=leaf)
    F = hs.hss_factor(dA, tree, compress=0)
    B = dg.random_rhs(A.n, 2, 1)
    Y = hs.hss_apply(F, torch.as_tensor(B, device="cuda")).cpu().numpy()
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx, leaf_max=leaf)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, compress=False)
    assert _rel(Y, oracle.apply(fac, B)) <= TOL
    Xd = np.linalg.solve(dg.bsr_to_dense(A), B)
    assert _rel(Y, Xd) <= 1e-9


APPROX = [("poisson", (16, 16), 1, 2, 64, 1e-6), ("helm", (16, 16), 2, 2, 64, 1e-4),
          ("helm", (24, 24), 2, 2, 64, 1e-6), ("poisson", (6, 6, 6), 1, 3, 64, 1e-5)]


@pytest.mark.parametrize("kind,n,p,dim,leaf,tol", APPROX)
def test_fronts_and_apply_match_oracle(kind, n, p, dim, leaf, tol):
    import torch
    hs = _hss()
    mesh, A = _setup(kind, n, p, dim)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((dim, tuple(n), p), dA, leaf_max=leaf)
    F = hs.hss_factor(dA, tree, tol=tol, seed=3, keep_schur=1)
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx, leaf_max=leaf)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=tol, seed=3, rmax=96)
    logs = {r["box"]: r for r in fac["log"]}
    compressed = 0
    for b in range(nd["nbox"]):
        if nd["nb"][b] == 0:
            continue
        S, H, kmax, r = F.export_front(b)
        assert _rel(S, fac["boxes"][b]["S"]) <= TOL, b
        rec = logs[b]
        if rec.get("nnodes", 1) > 1:
            compressed += 1
            assert kmax == rec["kmax"] and r == rec["r"], (b, kmax, rec["kmax"], r, rec["r"])
    assert compressed > 0
    X = dg.random_rhs(A.n, 2, 7)
    Y = hs.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy()
    assert _rel(Y, oracle.apply(fac, X)) <= TOL


def test_hss_approximant_matches_oracle():
    hs = _hss()
    mesh, A = _setup("helm", (16, 16), 2)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (16, 16), 2), dA)
    F = hs.hss_factor(dA, tree, tol=1e-4, seed=1, keep_schur=1)
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=1e-4, seed=1, rmax=96, keep_h=True)
    for b in (0, 1, 2, 3):
        S, H, kmax, r = F.export_front(b)
        assert _rel(H, fac["boxes"][b]["H"]) <= TOL
        assert _rel(H, S) <= 1e-2          # the approximant is close to S


def test_capped_sample_width_keeps_s_like_oracle():
    """With the sample width capped at 32 and a tight tolerance, fronts whose
    ranks exceed r - 10 keep S (H = S) on both sides; the rest are compressed
    as usual.  Same fronts, same H, same count."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (16, 16), 2)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (16, 16), 2), dA)
    F = hs.hss_factor(dA, tree, tol=1e-9, seed=2, rmax=32, keep_schur=1)
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=1e-9, seed=2, rmax=32, keep_h=True)
    capped = [r["box"] for r in fac["log"] if r.get("capped")]
    assert 0 < len(capped) < sum(1 for r in fac["log"] if r.get("nnodes", 1) > 1)
    assert F.info()["capped_fronts"] == len(capped)
    for b in range(nd["nbox"]):
        if nd["nb"][b] == 0:
            continue
        S, H, kmax, r = F.export_front(b)
        assert _rel(H, fac["boxes"][b]["H"]) <= TOL, b
        if b in capped:
            assert np.array_equal(H, S), b
    X = dg.random_rhs(A.n, 1, 4)
    Y = hs.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy()
    assert _rel(Y, oracle.apply(fac, X)) <= TOL


SOLVES = [("poisson", (16, 16), 1, 1e-6, 1e-10), ("helm", (32, 32), 2, 1e-4, 1e-8),
          ("helm", (16, 16), 3, 1e-5, 1e-8)]


@pytest.mark.parametrize("kind,n,p,tol,rtol", SOLVES)
def test_fgmres_matches_oracle(kind, n, p, tol, rtol):
    import torch
    hs = _hss()
    mesh, A = _setup(kind, n, p)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, tuple(n), p), dA)
    F = hs.hss_factor(dA, tree, tol=tol, seed=0)
    b = dg.point_source_rhs(mesh, 0)[:, 0] if kind == "helm" else dg.random_rhs(A.n, 1, 0)[:, 0]
    x, st = hs.fgmres_solve(dA, F, torch.as_tensor(b, device="cuda"), rtol=rtol, restart=30)
    Acsr = dg.bsr_to_csr(A)
    xr = x.cpu().numpy()
    assert st.converged and np.linalg.norm(b - Acsr @ xr) <= rtol * np.linalg.norm(b) * 1.0000001
    nd = oracle.nd_order(2, mesh.n, p, A.row_ptr, A.col_idx)
    fac = oracle.factor(Acsr, nd, tol=tol, seed=0, rmax=96)
    xo, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=rtol, restart=30)
    assert abs(st.iters - info["iters"]) <= max(1, round(0.1 * info["iters"]))
    assert _rel(xr, xo) <= 1e3 * rtol


def test_unpreconditioned_history_matches_oracle():
    import torch
    hs = _hss()
    mesh, A = _setup("poisson", (6, 6), 1)
    dA = hs.DeviceBSR.from_host(A)
    b = dg.random_rhs(A.n, 1, 2)[:, 0]
    x, st = hs.fgmres_solve(dA, None, torch.as_tensor(b, device="cuda"), restart=20, rtol=1e-9, maxit=20)
    h = hs.fgmres_history(0)
    Acsr = dg.bsr_to_csr(A)
    xo, info = oracle.fgmres(lambda v: Acsr @ v, None, b, restart=20, rtol=1e-9, maxit=20)
    assert len(h) == len(info["hist"]) == 20
    assert np.allclose(h, info["hist"], rtol=1e-8, atol=1e-15)
    assert not st.converged


def test_multiple_rhs_apply_and_solve():
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (16, 16), 2)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (16, 16), 2), dA)
    F = hs.hss_factor(dA, tree, tol=1e-4)
    B = torch.as_tensor(dg.random_rhs(A.n, 5, 3, kind="normal"), device="cuda")
    Y = hs.hss_apply(F, B)
    for k in range(5):
        yk = hs.hss_apply(F, B[:, k].contiguous())
        assert torch.allclose(Y[:, k], yk, rtol=1e-13, atol=1e-13)
    X, st = hs.fgmres_solve(dA, F, B, rtol=1e-8)
    assert st.converged
    R = B.cpu().numpy() - dg.bsr_to_csr(A) @ X.cpu().numpy()
    assert np.linalg.norm(R, axis=0).max() <= 1e-8 * np.linalg.norm(B.cpu().numpy(), axis=0).min() * 1.01


def test_errors_are_reported():
    import torch
    hs = _hss()
    mesh, A = _setup("poisson", (4, 4), 1)
    dA = hs.DeviceBSR.from_host(A)
    with pytest.raises(hs.HssError) as e:
        hs.nd_order((2, (5, 4), 1), dA)       # mesh and matrix disagree
    assert e.value.code == hs.HSS_EINVAL
    tree = hs.nd_order((2, (4, 4), 1), dA, leaf_max=8)
    with pytest.raises(hs.HssError) as e:
        hs.hss_factor(dA, tree, rmax=4096)
    assert e.value.code == hs.HSS_EINVAL
    # a zero block row makes a front singular
    A2 = dg.assemble_sipg(mesh)
    e0 = 5
    for t in range(A2.row_ptr[e0], A2.row_ptr[e0 + 1]):
        A2.val[t] = 0.0
    for e in range(A2.nb):
        for t in range(A2.row_ptr[e], A2.row_ptr[e + 1]):
            if A2.col_idx[t] == e0:
                A2.val[t] = 0.0
    dA2 = hs.DeviceBSR.from_host(A2)
    tree2 = hs.nd_order((2, (4, 4), 1), dA2, leaf_max=8)
    with pytest.raises(hs.HssError) as e:
        hs.hss_factor(dA2, tree2, compress=0)
    assert e.value.code == hs.HSS_ESINGULAR
    # non-convergence returns the iterate and the flag
    F = hs.hss_factor(dA, tree, compress=1, tol=1e-1)
    b = torch.as_tensor(dg.random_rhs(A.n, 1, 0)[:, 0], device="cuda")
    x, st = hs.fgmres_solve(dA, None, b, rtol=1e-14, maxit=2)
    assert not st.converged and st.iters == 2
    # a NaN or an infinite value anywhere in A is rejected (one stored value
    # in an off-diagonal block, then in the last block)
    for pos, bad in ((A.row_ptr[3] * A.bs * A.bs + 2, float("nan")), (A.val.size - 1, float("inf"))):
        A3 = dg.assemble_sipg(mesh)
        A3.val.reshape(-1)[pos] = bad
        dA3 = hs.DeviceBSR.from_host(A3)
        with pytest.raises(hs.HssError) as e:
            hs.hss_factor(dA3, tree)
        assert e.value.code == hs.HSS_EINVAL and "NaN or infinite" in str(e.value)
    # the same matrix without the bad value factors (the context is still usable)
    hs.hss_factor(dA, tree)


def test_tensor_core_wait_timeout_is_reported():
    """The tcgen05 kernel's bounded mbarrier wait: with its MMAs left out the
    barrier never completes, the wait gives up after the given number of polls
    and the call returns HSS_ETIMEOUT; the GPU stays usable (a tensor-core
    GEMM right after it is correct)."""
    import torch
    hs = _hss()
    assert hs.tc_timeout_selftest(1 << 10) == hs.HSS_ETIMEOUT
    assert "expired" in hs._lib.hss_last_error().decode()
    assert hs.tc_timeout_selftest(1 << 14) == hs.HSS_ETIMEOUT
    g = torch.Generator(device="cpu").manual_seed(3)
    A = torch.randn(256, 128, generator=g).cuda()
    B = torch.randn(128, 192, generator=g).cuda()
    C = hs.gemm_f32(A, B, engine=1)
    ref = A.double() @ B.double()
    assert (C.double() - ref).abs().max().item() <= 2e-6 * (A.double().abs() @ B.double().abs()).max().item()


@pytest.mark.parametrize("m,n,k", [(300, 200, 70), (128, 128, 32), (513, 77, 257), (64, 300, 5), (1, 1, 1),
                                   (300, 260, 132), (256, 512, 1024), (130, 132, 16), (129, 4, 20)])
def test_gemm_f32_engines(m, n, k):
    """The FP32 GEMM engines against an FP64 product: SIMT FMA and tcgen05
    TF32 with the hi/lo split at FP32 accuracy (threads staging the operands,
    engine 1, or TMA through the 3-stage ring, engine 3), single TF32 at TF32
    accuracy.  Engine 3 runs where the operands suit TMA (n and k multiples of
    4 here: the column-major operands of the row-major call have leading
    dimensions n and k), with ragged tiles and K chunks (k = 20, 132), one
    chunk (16) and a long ring (1024 = 64 chunks of 16); elsewhere it falls
    back to engine 1."""
    import torch
    hs = _hss()
    g = torch.Generator(device="cpu").manual_seed(m * 7 + n)
    A = torch.randn(m, k, generator=g).cuda()
    B = torch.randn(k, n, generator=g).cuda()
    C0 = torch.randn(m, n, generator=g).cuda()
    ref = (A.double() @ B.double()) * 0.5 + C0.double() * 2.0
    scale = (A.double().abs() @ B.double().abs()).max().item() + 1.0
    for engine, tol in ((0, 2e-6), (1, 2e-6), (2, 2e-3), (3, 2e-6)):
        C = C0.clone()
        hs.profile_reset()
        hs.profile_enable(True)
        hs.gemm_f32(A, B, C, alpha=0.5, beta=2.0, engine=engine)
        hs.profile_enable(False)
        cls = hs.profile_read()
        if engine == 3:
            assert ("gemm_tma" in cls) == (n % 4 == 0 and k % 4 == 0), (cls.keys(), n, k)
        torch.cuda.synchronize()
        err = (C.double() - ref).abs().max().item() / scale
        assert err <= tol, (engine, err)


@pytest.mark.parametrize("p", [2, 1])
def test_fp32_form_tensor_cores_match_simt(p):
    """The FP32 form with tcgen05 GEMMs (TF32 hi/lo split) against the same form
    with SIMT FMA GEMMs.  With compression off (pure arithmetic), both FP32
    Schur complements stay within the same order of the FP64 ones; with
    compression on, both solves converge alike.  p = 2 (9 dofs per element)
    runs the fronts whose size is not a multiple of 4 on the thread-staging
    kernel and the others on the TMA kernel; p = 1 (4 dofs per element: every
    front 16-byte aligned) runs all sampling products Y = S Omega and
    Z = S^t Psi on the TMA kernel (the profile shows which ran)."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (32, 32), p)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (32, 32), p), dA)
    F64 = hs.hss_factor(dA, tree, compress=0, keep_schur=1)
    Ft = hs.hss_factor(dA, tree, compress=0, precision="fp32", tensor_cores=1, keep_schur=1)
    Fs = hs.hss_factor(dA, tree, compress=0, precision="fp32", tensor_cores=0, keep_schur=1)
    ex = tree.export()
    big = [b for b in range(len(ex["nb"])) if ex["ni"][b] + ex["nb"][b] >= 128 and ex["nb"][b] > 0]
    assert big
    for b in big:
        S64, _, _, _ = F64.export_front(b)
        St, _, _, _ = Ft.export_front(b)
        Ss, _, _, _ = Fs.export_front(b)
        et, es = _rel(St, S64), _rel(Ss, S64)
        # the split drops the lo*lo product and the tensor core's internal sums are
        # not single-rounded FMAs: a few times the FMA-chain error, same order
        assert et <= 10.0 * es + 1e-6 and et <= 1e-2, (b, et, es)
    hs.profile_reset()
    hs.profile_enable(True)
    Ftc = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", tensor_cores=1, keep_schur=1)
    hs.profile_enable(False)
    cls = hs.profile_read()
    if p == 1:   # every front size is a multiple of 4 (p = 2: only those of 36 k dofs)
        assert any(k.startswith("gemm_tma") for k in cls) and "gemm_tc" not in cls, cls.keys()
    Fsi = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", tensor_cores=0, keep_schur=1)
    # same ranks and widths from the two engines' samples, approximants of the same quality
    lt, ls = Ftc.export_log(), Fsi.export_log()
    assert (np.abs(lt["kmax"] - ls["kmax"]) <= 1).all() and (lt["r"] == ls["r"]).mean() >= 0.99
    for b in big:
        St, Ht, _, _ = Ftc.export_front(b)
        Ss, Hs_, _, _ = Fsi.export_front(b)
        assert _rel(Ht, St) <= 10.0 * _rel(Hs_, Ss) + 1e-5, b
    bvec = torch.as_tensor(dg.point_source_rhs(mesh, 0)[:, 0], device="cuda")
    xt, st = hs.fgmres_solve(dA, Ftc, bvec, rtol=1e-8)
    xs, ss = hs.fgmres_solve(dA, Fsi, bvec, rtol=1e-8)
    assert st.converged and ss.converged and abs(st.iters - ss.iters) <= 2


def test_gemm_engine_tuner_times_once_and_matches_simt():
    """tensor_cores = 3: the first factorization times each GEMM shape class
    on SIMT and on the tcgen05 split kernel and keeps the faster; a second
    factorization of the same structure reuses every choice (no timing, same
    engine split).  The result has the accuracy of the SIMT form: same widths
    (ranks within one), approximants of the same quality, FGMRES alike."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (48, 48), 1)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (48, 48), 1), dA)
    F1 = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", tensor_cores=3, keep_schur=1)
    F2 = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", tensor_cores=3, keep_schur=1)
    Fs = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", tensor_cores=0, keep_schur=1)
    i1, i2, i0 = F1.info(), F2.info(), Fs.info()
    print(f"\nengine split (SIMT, TMA, staged): {i1['gemm_simt']}, {i1['gemm_tma']}, {i1['gemm_staged']}; "
          f"timed {i1['gemm_timed']} then {i2['gemm_timed']}")
    assert i2["gemm_timed"] == 0
    assert (i1["gemm_simt"], i1["gemm_tma"], i1["gemm_staged"]) == (i2["gemm_simt"], i2["gemm_tma"],
                                                                   i2["gemm_staged"])
    assert i0["gemm_tma"] == 0 and i0["gemm_staged"] == 0
    l1, l0 = F1.export_log(), Fs.export_log()
    assert (np.abs(l1["kmax"] - l0["kmax"]) <= 1).all() and (l1["r"] == l0["r"]).mean() >= 0.99
    ex = tree.export()
    for b in range(len(ex["nb"])):
        if ex["nb"][b] >= 128:
            S1, H1, _, _ = F1.export_front(b)
            S0, H0, _, _ = Fs.export_front(b)
            assert _rel(H1, S1) <= 10.0 * _rel(H0, S0) + 1e-5, b
    bvec = torch.as_tensor(dg.point_source_rhs(mesh, 0)[:, 0], device="cuda")
    _, s1 = hs.fgmres_solve(dA, F1, bvec, rtol=1e-8)
    _, s0 = hs.fgmres_solve(dA, Fs, bvec, rtol=1e-8)
    assert s1.converged and s0.converged and abs(s1.iters - s0.iters) <= 2


def test_bf16_sampling_matches_fp32_sampling():
    """sample_bf16 = 1: the sampling products of the 16-byte aligned fronts
    (|B| >= 128) run on tcgen05 kind::f16 with S in three BF16 terms (about
    FP32 accuracy; the +-1 matrix is exact in BF16).  Against the same FP32
    form with SIMT sampling: the same widths, largest ranks within one,
    approximants of the same quality against the oracle's (the compression of
    the oracle's own S through hss_front_compress), and FGMRES alike."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (32, 32), 1)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (32, 32), 1), dA)
    Fb = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", sample_bf16=1, keep_schur=1)
    Fs = hs.hss_factor(dA, tree, tol=1e-4, precision="fp32", keep_schur=1)
    ib = Fb.info()
    assert ib["gemm_bf16"] > 0 and Fs.info()["gemm_bf16"] == 0
    lb, ls = Fb.export_log(), Fs.export_log()
    assert (np.abs(lb["kmax"] - ls["kmax"]) <= 1).all() and (lb["r"] == ls["r"]).mean() >= 0.99
    nd = oracle.nd_order(2, mesh.n, 1, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=1e-4, seed=0, rmax=96, keep_h=True)
    checked = 0
    for b in range(int(nd["nbox"])):
        if nd["nb"][b] < 128:
            continue
        S = fac["boxes"][b]["S"]
        Hb = hs.front_compress(tree, b, S, tol=1e-4, seed=0, rmax=96, precision="fp32", sample_bf16=1)[0]
        Hs_ = hs.front_compress(tree, b, S, tol=1e-4, seed=0, rmax=96, precision="fp32")[0]
        eb, es = _rel(Hb, fac["boxes"][b]["H"]), _rel(Hs_, fac["boxes"][b]["H"])
        assert eb <= 10.0 * es + 1e-5, (b, eb, es)
        checked += 1
    assert checked > 0
    bvec = torch.as_tensor(dg.point_source_rhs(mesh, 0)[:, 0], device="cuda")
    _, sb = hs.fgmres_solve(dA, Fb, bvec, rtol=1e-8)
    _, ss = hs.fgmres_solve(dA, Fs, bvec, rtol=1e-8)
    assert sb.converged and ss.converged and abs(sb.iters - ss.iters) <= 2


def test_autotuned_apply_matches_oracle_and_is_cached():
    """The tuned work split (columns per apply work item, per stage and
    direction) changes only the summation order: the apply still matches the
    oracle to 1e-10 and the untuned apply to 1e-13; a second factorization of
    the same structure reuses the cached choice."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (24, 24), 2)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (24, 24), 2), dA)
    F0 = hs.hss_factor(dA, tree, tol=1e-6, seed=3)
    F1 = hs.hss_factor(dA, tree, tol=1e-6, seed=3, autotune=1)
    F2 = hs.hss_factor(dA, tree, tol=1e-6, seed=4, autotune=1)
    p0, p1, p2 = F0.apply_plan(), F1.apply_plan(), F2.apply_plan()
    assert (p0[0] == 64).all() and (p0[1] == 64).all()
    assert set(p1[0].tolist() + p1[1].tolist()) <= {32, 64, 128, 256}
    assert np.array_equal(p1[0], p2[0]) and np.array_equal(p1[1], p2[1])
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=1e-6, seed=3, rmax=96)
    X = dg.random_rhs(A.n, 3, 5)
    for k in (1, 3):
        Xk = torch.as_tensor(np.asfortranarray(X[:, :k]), device="cuda")
        Y0 = hs.hss_apply(F0, Xk).cpu().numpy().reshape(A.n, k)
        Y1 = hs.hss_apply(F1, Xk).cpu().numpy().reshape(A.n, k)
        assert _rel(Y1, oracle.apply(fac, X[:, :k])) <= TOL
        assert _rel(Y1, Y0) <= 1e-13


@pytest.mark.parametrize("oversample,r0,regrows", [(10, 32, False), (0, 8, True)])
def test_residual_probe_matches_oracle(oversample, r0, regrows):
    """The residual probe of accepted approximants (4 +-1 vectors, threshold
    10 tol depth): with oversampling 10 no front fails it and nothing changes;
    with none, fronts fail, sample again, and the GPU takes the same decisions
    as the oracle (same rounds per front, same regrowth count, H and apply
    within 1e-10)."""
    import torch
    hs = _hss()
    mesh, A = _setup("helm", (16, 16), 2)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (16, 16), 2), dA)
    kw = dict(tol=1e-6, seed=1, r0=r0, rmax=96, oversample=oversample)
    F = hs.hss_factor(dA, tree, probe=4, keep_schur=1, **kw)
    F0 = hs.hss_factor(dA, tree, keep_schur=1, **kw)
    nd = oracle.nd_order(2, mesh.n, 2, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, probe=4, keep_h=True, **kw)
    regrown = sum(r.get("probe_regrown", 0) for r in fac["log"])
    assert (regrown > 0) == regrows
    assert F.info()["probe_regrown"] == regrown and F0.info()["probe_regrown"] == 0
    lg = F.export_log()
    gpu_rounds = dict(zip(lg["box"].tolist(), lg["rounds"].tolist()))
    for rec in fac["log"]:
        if rec.get("nnodes", 1) > 1:
            assert gpu_rounds[rec["box"]] == rec["rounds"], rec["box"]
    for b in range(nd["nbox"]):
        if nd["nb"][b] == 0:
            continue
        _, H, _, _ = F.export_front(b)
        assert _rel(H, fac["boxes"][b]["H"]) <= TOL, b
        if not regrows:
            assert np.array_equal(H, F0.export_front(b)[1])
    X = dg.random_rhs(A.n, 1, 2)
    Y = hs.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy().reshape(A.n, 1)
    assert _rel(Y, oracle.apply(fac, X)) <= TOL
