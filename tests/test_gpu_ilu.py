"""Block ILU(0), the comparison preconditioner of Sec. 5, through the C ABI
against the oracle (oracle/ilu.py).

Bars: factor and apply within 1e-10 relative of the oracle in FP64 (the GPU
multiplies by explicit U_kk^-1 where the oracle solves; both are backward
stable, and the small diagonal blocks keep the difference near 1e-14); exact
on a block-tridiagonal chain; FGMRES iteration counts within +-10% (at least
+-1) of the oracle's with the same preconditioner.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import ilu as oilu
from paper_1508_07798_gb300 import dg_inputs as dg

pytestmark = pytest.mark.gpu


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [((16, 16), 1, "poisson"), ((12, 12), 2, "helm"), ((7, 5), 3, "poisson"), ((4, 4, 4), 1, "poisson"),
         ((3, 3, 2), 3, "poisson")]


def _matrix(n, p, kind):
    mesh = dg.Mesh(len(n), tuple(n) + (1,) * (3 - len(n)), p)
    if kind == "helm":
        return mesh, dg.assemble_sipg(mesh, c_elem=dg.cosine_field(mesh, 0), kappa=dg.helmholtz_kappa(n[0], p))
    return mesh, dg.assemble_sipg(mesh)


@pytest.mark.parametrize("n,p,kind", CASES)
def test_apply_matches_oracle(n, p, kind):
    """Several levels per sweep, ragged level sizes; bs from 4 to 64 (the 3D
    p = 3 case takes two lanes per component and 97 KB of shared memory)."""
    import torch
    hs = _hss()
    mesh, A = _matrix(n, p, kind)
    M = hs.ilu0_factor(hs.DeviceBSR.from_host(A))
    ref = oilu.ilu0(A.row_ptr, A.col_idx, A.val)
    for k in (1, 3, 9):
        X = dg.random_rhs(A.n, k, 10 + k)
        Y = hs.ilu0_apply(M, torch.as_tensor(X, device="cuda")).cpu().numpy().reshape(A.n, k)
        assert _rel(Y, oilu.ilu0_apply(ref, X)) <= 1e-10, k


def test_chain_is_exact_and_apply_in_place():
    import torch
    hs = _hss()
    mesh = dg.Mesh(2, (9, 1, 1), 2)
    A = dg.assemble_sipg(mesh)
    M = hs.ilu0_factor(hs.DeviceBSR.from_host(A))
    X = dg.random_rhs(A.n, 2, 0)
    xd = torch.as_tensor(np.asfortranarray(X), device="cuda").t().contiguous()   # column-major storage
    hs._check(hs._lib.ilu0_apply(M.h, 2, hs._ptr(xd), A.n, hs._ptr(xd), A.n, hs._stream()))
    Y = xd.t().cpu().numpy()
    assert _rel(Y, np.linalg.solve(dg.bsr_to_dense(A), X)) <= 1e-12


def test_fgmres_with_ilu0_matches_oracle():
    import torch
    hs = _hss()
    mesh, A = _matrix((16, 16), 1, "poisson")
    Acsr = dg.bsr_to_csr(A)
    b = dg.random_rhs(A.n, 1, 0)[:, 0]
    dA = hs.DeviceBSR.from_host(A)
    M = hs.ilu0_factor(dA)
    x, st = hs.fgmres_solve(dA, M, torch.as_tensor(b, device="cuda"), rtol=1e-8, maxit=3000)
    ref = oilu.ilu0(A.row_ptr, A.col_idx, A.val)
    _, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oilu.ilu0_apply(ref, v), b, rtol=1e-8, maxit=3000)
    assert st.converged and info["converged"]
    assert abs(st.iters - info["iters"]) <= max(1, round(0.1 * info["iters"])), (st.iters, info["iters"])
    xr = x.cpu().numpy()
    assert np.linalg.norm(b - Acsr @ xr) <= 1e-8 * np.linalg.norm(b) * 1.0000001
    # several right-hand sides: lock-step processes with the same preconditioner
    B = dg.random_rhs(A.n, 3, 1)
    X3, st3 = hs.fgmres_solve(dA, M, torch.as_tensor(B, device="cuda"), rtol=1e-8, maxit=3000)
    R = B - Acsr @ X3.cpu().numpy().reshape(A.n, 3)
    assert st3.converged and (np.linalg.norm(R, axis=0) <= 1e-8 * np.linalg.norm(B, axis=0) * 1.0000001).all()


def test_errors_are_reported():
    import torch
    hs = _hss()
    mesh, A = _matrix((4, 4), 1, "poisson")
    # a zero diagonal block in row 0: U_00 is singular
    val = A.val.copy()
    d0 = list(A.col_idx[A.row_ptr[0]:A.row_ptr[1]]).index(0)
    val[A.row_ptr[0] + d0] = 0.0
    Az = dg.BSR(nb=A.nb, bs=A.bs, row_ptr=A.row_ptr, col_idx=A.col_idx, val=val, meta=A.meta)
    with pytest.raises(hs.HssError) as e:
        hs.ilu0_factor(hs.DeviceBSR.from_host(Az))
    assert e.value.code == hs.HSS_ESINGULAR and "block row 0" in str(e.value)
    # a block row without its diagonal block
    keep = np.ones(A.nnzb, bool)
    keep[A.row_ptr[5] + list(A.col_idx[A.row_ptr[5]:A.row_ptr[6]]).index(5)] = False
    rp = np.concatenate([[0], np.cumsum([keep[A.row_ptr[i]:A.row_ptr[i + 1]].sum() for i in range(A.nb)])])
    An = dg.BSR(nb=A.nb, bs=A.bs, row_ptr=rp.astype(np.int32), col_idx=A.col_idx[keep].copy(),
                val=np.ascontiguousarray(A.val[keep]), meta=A.meta)
    with pytest.raises(hs.HssError) as e:
        hs.ilu0_factor(hs.DeviceBSR.from_host(An))
    assert e.value.code == hs.HSS_EINVAL and "no diagonal block" in str(e.value)
    out = ctypes.c_void_p()
    assert hs._lib.ilu0_factor(None, None, ctypes.byref(out)) == hs.HSS_EINVAL
    assert hs._lib.ilu0_apply(None, 1, None, 1, None, 1, None) == hs.HSS_EINVAL
    dA = hs.DeviceBSR.from_host(A)
    M = hs.ilu0_factor(dA)
    b = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x, st = hs.fgmres_solve(dA, M, b)
    assert st.converged and st.iters == 0 and float(x.abs().max()) == 0.0


def test_ilu_iterations_grow_with_n_while_hss_stays_flat():
    """Sec. 5, Poisson: the HSS preconditioner's GMRES iterations do not grow
    under h-refinement, ILU(0)'s do."""
    import torch
    hs = _hss()
    rows = []
    for n in (16, 32, 64):
        mesh, A = _matrix((n, n), 1, "poisson")
        dA = hs.DeviceBSR.from_host(A)
        b = torch.as_tensor(dg.random_rhs(A.n, 1, 0)[:, 0], device="cuda")
        _, si = hs.fgmres_solve(dA, hs.ilu0_factor(dA), b, rtol=1e-8, maxit=5000)
        tree = hs.nd_order((2, (n, n), 1), dA)
        _, sh = hs.fgmres_solve(dA, hs.hss_factor(dA, tree, tol=1e-6), b, rtol=1e-8)
        assert si.converged and sh.converged
        rows.append((n, si.iters, sh.iters))
    print("\nPoisson p=1, GMRES(30) iterations to 1e-8 (n, ILU(0), HSS):", rows)
    assert rows[1][1] >= 1.5 * rows[0][1] and rows[2][1] >= 1.5 * rows[1][1]
    assert max(r[2] for r in rows) - min(r[2] for r in rows) <= 1
