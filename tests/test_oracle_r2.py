"""Oracle pins for the structured merge (reading R2, oracle/merge.py):
Algorithm 1's block solve of eq. (37) with the second Schur complement
compressed, and Algorithm 3 for the top block."""
import numpy as np
import pytest

import oracle
from oracle import merge as omerge
from paper_1508_07798_gb300 import dg_inputs as dg


def _problem(kind, n, p, dim=2):
    mesh = dg.Mesh(dim, tuple(n) + (1,) * (3 - dim), p)
    if kind == "helm":
        A = dg.assemble_sipg(mesh, c_elem=dg.cosine_field(mesh, 0), kappa=dg.helmholtz_kappa(n[0], p))
    else:
        A = dg.assemble_sipg(mesh)
    nd = oracle.nd_order(dim, mesh.n, p, A.row_ptr, A.col_idx)
    return mesh, A, nd, dg.bsr_to_csr(A)


def test_block_solve_without_compression_is_the_inverse():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((40, 40)) + 40 * np.eye(40)
    for n1 in (0, 1, 17, 40):
        X, info = omerge.block_inverse(M, n1, None, 1e-6, 0, 0)
        assert np.abs(X @ M - np.eye(40)).max() <= 1e-12
        # S~ is the Schur complement of the leading block: the inverse of the trailing block of M^-1
        if 0 < n1 < 40:
            assert np.allclose(info["St"], np.linalg.inv(np.linalg.inv(M)[n1:, n1:]), atol=1e-10)


@pytest.mark.parametrize("kind,n,p,tol", [("poisson", (16, 16), 1, 1e-4), ("helm", (16, 16), 2, 1e-4),
                                         ("helm", (12, 12), 3, 1e-6)])
def test_structured_inverse_is_exact_for_the_perturbed_block(kind, n, p, tol):
    """Written as a matrix, eq. (37) with H~ in place of S~ is the exact
    inverse of A_ii + blockdiag(0, H~ - S~): a closed-form identity for every
    parent front and for the top block (Algorithm 3)."""
    mesh, A, nd, Acsr = _problem(kind, n, p)
    fac = oracle.factor(Acsr, nd, tol=tol, seed=2, rmax=96, merge="structured")
    checked, compressed = 0, 0
    for rec in fac["log"]:
        b = rec["box"]
        if "tilde" not in rec:
            continue
        F, X = fac["boxes"][b]["F"], fac["boxes"][b]["Xinv"]
        ni = rec["ni"]
        n1, _ = omerge.interior_split(nd, b)
        P = F[:ni, :ni].copy()
        P[n1:, n1:] += rec["tilde"]["Ht"] - rec["tilde"]["St"]
        assert np.abs(X @ P - np.eye(ni)).max() <= 1e-8, b
        checked += 1
        compressed += rec["tilde"]["rep"] is not None
    ti = fac["top_info"]
    P0 = fac["A0"].copy()
    n0 = nd["bset"][0].size
    P0[n0:, n0:] += ti["Ht"] - ti["St"]
    assert np.abs(fac["top_inv"] @ P0 - np.eye(P0.shape[0])).max() <= 1e-8
    assert checked > 0 and compressed > 0 and ti["rep"] is not None


def test_interior_split_matches_the_child_ranges():
    mesh, A, nd, _ = _problem("poisson", (8, 6), 2)
    pos = np.empty(nd["dfs_dof"].size, dtype=np.int64)
    pos[nd["dfs_dof"]] = np.arange(nd["dfs_dof"].size)
    for b in range(nd["nbox"]):
        if nd["is_leaf"][b] or nd["iset"][b].size == 0:
            continue
        mu, nu = (int(c) for c in nd["child"][b])
        n1, dofs2 = omerge.interior_split(nd, b)
        I = nd["iset"][b]
        in_mu = (pos[I] >= nd["pos0"][mu]) & (pos[I] < nd["pos1"][mu])
        assert n1 == in_mu.sum() and in_mu[:n1].all()
        assert np.array_equal(dofs2, I[n1:])
        nodes = oracle.hss_tree_for_front(nd, nu, dofs2)
        if nodes:
            leaves = sorted((x["lo"], x["hi"]) for x in nodes if not x["children"])
            assert leaves[0][0] == 0 and leaves[-1][1] == dofs2.size
            assert all(a[1] == b_[0] for a, b_ in zip(leaves, leaves[1:]))


@pytest.mark.parametrize("kind,n,p,dim,tol", [("poisson", (16, 16), 1, 2, 1e-6), ("helm", (16, 16), 2, 2, 1e-4),
                                             ("poisson", (4, 4, 4), 1, 3, 1e-5)])
def test_structured_preconditioner_converges_like_dense_merge(kind, n, p, dim, tol):
    mesh, A, nd, Acsr = _problem(kind, n, p, dim)
    b = dg.random_rhs(A.n, 1, 0)[:, 0]
    its = {}
    for merge in ("dense", "structured"):
        fac = oracle.factor(Acsr, nd, tol=tol, seed=0, rmax=96, merge=merge)
        x, info = oracle.fgmres(lambda v: Acsr @ v, lambda v: oracle.apply(fac, v), b, rtol=1e-8, maxit=300)
        assert info["converged"] and np.linalg.norm(b - Acsr @ x) <= 1e-8 * np.linalg.norm(b) * 1.0000001
        its[merge] = info["iters"]
    assert abs(its["structured"] - its["dense"]) <= 1, its


def test_structured_merge_with_compression_off_is_exact():
    mesh, A, nd, Acsr = _problem("helm", (10, 10), 2)
    fac = oracle.factor(Acsr, nd, compress=False, merge="structured")
    X = dg.random_rhs(A.n, 2, 1)
    Z = oracle.apply(fac, X)
    assert np.linalg.norm(Z - np.linalg.solve(Acsr.toarray(), X)) <= 1e-10 * np.linalg.norm(Z)
    with pytest.raises(ValueError):
        oracle.factor(Acsr, nd, merge="fast")
