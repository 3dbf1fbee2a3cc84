"""The structured merge (reading R2: Algorithm 1's block solve of eq. (37)
with the second Schur complement compressed, Algorithm 3 for the top block)
on the GPU (hss_factor_opts.merge = 1) against the oracle's
factor(merge="structured"), through the C ABI.

FP64, the cases of the oracle's own R2 pins: every front's Schur complement S
(which now depends on the approximate interior inverse) and its approximant H
within 1e-10, norm-wise and element-wise; the apply (which uses the perturbed
interior inverses) within 1e-10; FGMRES iterations within +-10% (at least
+-1) of the oracle's with its structured factor, and within two of the GPU's
own R1 factorization."""
import numpy as np
import pytest

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg
from parity import rel_fro, rel_max

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _problem(kind, n, p, dim=2):
    mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
    if kind == "helm":
        A = dg.assemble_sipg(mesh, c_elem=dg.cosine_field(mesh, 0), kappa=dg.helmholtz_kappa(n[0], p))
    else:
        A = dg.assemble_sipg(mesh)
    return mesh, A


@pytest.mark.parametrize("kind,n,p,tol,dim", [("poisson", (16, 16), 1, 1e-4, 2), ("helm", (16, 16), 2, 1e-4, 2),
                                             ("helm", (12, 12), 3, 1e-6, 2), ("poisson", (6, 6, 6), 1, 1e-4, 3)])
def test_structured_merge_matches_oracle(kind, n, p, tol, dim):
    import torch
    from paper_1508_07798_gb300 import hssnd as hs
    mesh, A = _problem(kind, n, p, dim)
    Acsr = dg.bsr_to_csr(A)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((dim, tuple(n), p), dA)
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx)
    fac = oracle.factor(Acsr, nd, tol=tol, seed=2, rmax=96, merge="structured", keep_h=True)
    F = hs.hss_factor(dA, tree, tol=tol, seed=2, rmax=96, merge=1, keep_schur=1)
    worst = dict(S=0.0, H=0.0, Smax=0.0, Hmax=0.0)
    structured = 0
    for b in range(int(nd["nbox"])):
        if nd["nb"][b] == 0:
            continue
        S, H, _, _ = F.export_front(b)
        worst["S"] = max(worst["S"], rel_fro(S, fac["boxes"][b]["S"]))
        worst["H"] = max(worst["H"], rel_fro(H, fac["boxes"][b]["H"]))
        worst["Smax"] = max(worst["Smax"], rel_max(S, fac["boxes"][b]["S"]))
        worst["Hmax"] = max(worst["Hmax"], rel_max(H, fac["boxes"][b]["H"]))
        structured += fac["boxes"][b].get("Xinv") is not None
    X = dg.random_rhs(A.n, 2, 3)
    Y = hs.hss_apply(F, torch.as_tensor(X, device="cuda")).cpu().numpy()
    Yo = oracle.apply(fac, X)
    ea = rel_fro(Y, Yo)
    print(f"\n{kind} {n} p={p}: {structured} structured fronts; S {worst['S']:.2e} / {worst['Smax']:.2e}, "
          f"H {worst['H']:.2e} / {worst['Hmax']:.2e}, apply {ea:.2e}")
    assert structured > 0
    assert max(worst.values()) <= TOL and ea <= TOL and rel_max(Y, Yo) <= TOL
    b = X[:, 0]
    _, io = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8, restart=30)
    x, st = hs.fgmres_solve(dA, F, torch.as_tensor(b, device="cuda"), rtol=1e-8, restart=30)
    res = np.linalg.norm(b - Acsr @ x.cpu().numpy()) / np.linalg.norm(b)
    F1 = hs.hss_factor(dA, tree, tol=tol, seed=2, rmax=96)
    _, s1 = hs.fgmres_solve(dA, F1, torch.as_tensor(b, device="cuda"), rtol=1e-8, restart=30)
    print(f"FGMRES: R2 GPU {st.iters}, R2 oracle {io['iters']}, R1 GPU {s1.iters}; residual {res:.2e}")
    assert st.converged and res <= 1e-8 * (1 + 1e-6)
    assert abs(st.iters - io["iters"]) <= max(1, round(0.1 * io["iters"]))
    assert abs(st.iters - s1.iters) <= 2


def test_structured_merge_option_checks():
    """merge = 1 refuses the residual probe (the probe compares S with H in the
    parent front, and S~ is overwritten in place) and the batched form."""
    from paper_1508_07798_gb300 import hssnd as hs
    mesh, A = _problem("poisson", (8, 8), 1)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (8, 8), 1), dA)
    with pytest.raises(hs.HssError) as e:
        hs.hss_factor(dA, tree, merge=1, probe=4)
    assert e.value.code == hs.HSS_EINVAL
    forest = hs.nd_order_batched([(2, (8, 8), 1)], [dA])
    with pytest.raises(hs.HssError) as e:
        hs.hss_factor_batched([dA], forest, merge=1)
    assert e.value.code == hs.HSS_EINVAL
