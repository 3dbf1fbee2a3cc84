"""Rank structure of the Schur complements (Sec. 5, the rank studies of the
Laplace and Helmholtz operators) from the factor's rank log.

For the first box of each level (the lowest box id) the HSS rank k of its
Schur complement (largest ID rank over the HSS nodes, tol 1e-6):
* equals the oracle's on small meshes (same boxes, same |B|, same k);
* Laplace, h-refinement: k is nearly independent of N (p = 1, 32^2 .. 256^2
  elements: |B| grows 8x, k by at most 1.5x);
* Laplace, p-enrichment: k grows roughly as the square root of |B|
  (16^2 elements, p = 1..3: k / sqrt(|B|) stays within [1.2, 2]);
* Helmholtz (10 dofs per wavelength) against Laplace: larger ranks at the
  top level, a smaller gap further down the tree.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1508_07798_gb300 import dg_inputs as dg

pytestmark = pytest.mark.gpu


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def _matrix(kind, n, p):
    mesh = dg.Mesh(2, (n, n, 1), p)
    if kind == "poisson":
        return mesh, dg.assemble_sipg(mesh)
    return mesh, dg.assemble_sipg(mesh, kappa=dg.helmholtz_kappa(n, p))


def _gpu_ranks(kind, n, p, tol=1e-6):
    hs = _hss()
    mesh, A = _matrix(kind, n, p)
    dA = hs.DeviceBSR.from_host(A)
    tree = hs.nd_order((2, (n, n), p), dA)
    F = hs.hss_factor(dA, tree, tol=tol, seed=0, rmax=128)
    ex = tree.export()
    lg = F.export_log()
    k = dict(zip(lg["box"].tolist(), lg["kmax"].tolist()))
    out = {}
    for b in sorted(k):
        lev = int(ex["level"][b])
        if lev not in out and k[b] > 0:
            out[lev] = (b, int(ex["nb"][b]), k[b])
    return out


def _oracle_ranks(kind, n, p, tol=1e-6):
    mesh, A = _matrix(kind, n, p)
    nd = oracle.nd_order(2, mesh.n, p, A.row_ptr, A.col_idx)
    fac = oracle.factor(dg.bsr_to_csr(A), nd, tol=tol, seed=0, rmax=128)
    out = {}
    for rec in sorted(fac["log"], key=lambda r: r["box"]):
        if rec["level"] not in out and rec.get("kmax", 0) > 0:
            out[rec["level"]] = (rec["box"], rec["nb"], rec["kmax"])
    return out


@pytest.mark.parametrize("kind,n,p", [("poisson", 16, 1), ("poisson", 32, 1), ("poisson", 16, 2), ("helm", 32, 1)])
def test_first_box_ranks_match_oracle(kind, n, p):
    assert _gpu_ranks(kind, n, p) == _oracle_ranks(kind, n, p)


def test_laplace_ranks_under_h_and_p_refinement():
    h = {n: _gpu_ranks("poisson", n, 1)[1] for n in (32, 64, 128, 256)}
    pe = {p: _gpu_ranks("poisson", 16, p)[1] for p in (1, 2, 3)}
    print("\nLaplace, first top-level box: (box, |B|, k)")
    print("  h-refinement, p=1:", {f"{n}x{n}": v for n, v in h.items()})
    print("  p-enrichment, 16x16:", {f"p={p}": v for p, v in pe.items()},
          " k/sqrt|B|:", [round(v[2] / math.sqrt(v[1]), 2) for v in pe.values()])
    assert h[256][1] == 8 * h[32][1]
    assert h[256][2] <= 1.5 * h[32][2]
    ks = [pe[p][2] for p in (1, 2, 3)]
    assert ks[0] < ks[1] < ks[2]
    for v in pe.values():
        assert 1.2 <= v[2] / math.sqrt(v[1]) <= 2.0


def test_helmholtz_gap_shrinks_down_the_tree():
    lap, hel = _gpu_ranks("poisson", 64, 1), _gpu_ranks("helm", 64, 1)
    ratio = {lev: hel[lev][2] / lap[lev][2] for lev in sorted(lap) if lev in hel}
    print("\nHelmholtz / Laplace rank ratio by level (64x64, p=1):", {k: round(v, 2) for k, v in ratio.items()})
    assert ratio[1] > 1.0
    deep = max(lev for lev in ratio if lap[lev][1] >= 64)
    assert ratio[deep] < ratio[1]
