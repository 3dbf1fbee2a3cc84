"""Oracle pins for the interpolative decomposition and the HSS construction
(paper Sec. 2, Theorem 1, eq. (43) and its footnote)."""
import os

import numpy as np
import pytest

import oracle
from oracle.idecomp import interp_decomp
from oracle.hss import hss_compress
from oracle.rademacher import rademacher, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    C0 = 0x9E3779B97F4A7C15
    got = [int(splitmix64(np.uint64((k * C0) % 2 ** 64))) for k in range(len(vals))]
    assert got == vals


def test_rademacher_prefix_and_balance():
    a = rademacher(5, 0, 17, np.arange(300), np.arange(32))
    b = rademacher(5, 0, 17, np.arange(300), np.arange(64))
    assert np.array_equal(a, b[:, :32])
    assert set(np.unique(b)) == {-1.0, 1.0}
    assert abs(b.mean()) < 0.05
    c = rademacher(5, 1, 17, np.arange(300), np.arange(64))
    assert not np.array_equal(b, c)


def _with_spectrum(m, r, s, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    V, _ = np.linalg.qr(rng.standard_normal((r, len(s))))
    return (U * s) @ V.T


@pytest.mark.parametrize("m,r,tol", [(60, 40, 1e-6), (120, 50, 1e-4), (30, 64, 1e-8)])
def test_id_error_within_rrqr_bound(m, r, tol):
    s = 10.0 ** (-np.arange(min(m, r)) / 3.0)
    M = _with_spectrum(m, r, s, 1)
    U, J, T, info = interp_decomp(M, tol)
    k = info["k"]
    assert np.abs(T).max(initial=0.0) <= 2.0 + 1e-12            # footnote: |P| <= 2
    assert np.allclose(U[J], np.eye(k))                          # identity on the skeleton
    err = np.linalg.norm(M - U @ M[J], 2)
    sk = s[k] if k < s.size else 0.0
    assert err <= np.sqrt(1.0 + 4.0 * k * (m - k)) * sk * (1 + 1e-8) + 1e-14
    # the rank cut stops where the pivots fall below tol * |R_11|
    assert s[k - 1] > 0.1 * tol * s[0]
    assert err <= 10.0 * np.sqrt(1.0 + 4.0 * k * (m - k)) * tol * s[0]


def test_id_exact_rank_and_zero():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((50, 7)) @ rng.standard_normal((7, 40))
    U, J, T, info = interp_decomp(M, 1e-12)
    assert info["k"] == 7
    assert np.linalg.norm(M - U @ M[J]) <= 1e-11 * np.linalg.norm(M)
    U0, J0, T0, i0 = interp_decomp(np.zeros((10, 5)), 1e-6)
    assert i0["k"] == 0 and U0.shape == (10, 0)


def test_id_exchanges_enforce_bound():
    """Kahan's matrix defeats plain column pivoting; the exchange pass must
    still bring every interpolation coefficient to |T| <= 2."""
    n = 40
    c = 0.285
    s = np.sqrt(1 - c * c)
    R = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    K = np.diag(s ** np.arange(n)) @ R
    K = K @ np.diag(1.0 - 1e-8 * np.arange(n))      # keep the pivot order unchanged
    tol = s ** (n - 1.5)                               # rank cut at k = n - 1
    U, J, T, info = interp_decomp(K.T, tol)           # rows of K^t = columns of K
    assert info["k"] == n - 1
    assert info["swaps"] > 0
    assert np.abs(T).max() <= 2.0 + 1e-12
    M = K.T
    assert np.linalg.norm(M - U @ M[J], 2) <= np.sqrt(1 + 4.0 * (n - 1)) * np.linalg.svd(M, compute_uv=False)[-1] * 1.0001


def _nodes_binary(n, leaf):
    """Balanced binary HSS tree over range(n): list in post-order, root last."""
    nodes = []

    def build(lo, hi, depth):
        if hi - lo <= leaf:
            nodes.append(dict(lo=lo, hi=hi, children=[], depth=depth))
            return len(nodes) - 1
        mid = (lo + hi) // 2
        a = build(lo, mid, depth + 1)
        b = build(mid, hi, depth + 1)
        nodes.append(dict(lo=lo, hi=hi, children=[a, b], depth=depth))
        return len(nodes) - 1

    build(0, n, 0)
    return nodes


def _hss_by_construction(nodes, k, rng):
    """Random HSS matrix with nested bases of rank k (Sec. 2 definition)."""
    n = nodes[-1]["hi"]
    Ut, Vt = {}, {}
    for t, nd_ in enumerate(nodes[:-1]):
        if not nd_["children"]:
            m = nd_["hi"] - nd_["lo"]
            Ut[t] = rng.standard_normal((m, k))
            Vt[t] = rng.standard_normal((m, k))
        else:
            a, b = nd_["children"]
            Us = rng.standard_normal((2 * k, k))
            Vs = rng.standard_normal((2 * k, k))
            Ut[t] = np.vstack([Ut[a] @ Us[:k], Ut[b] @ Us[k:]])
            Vt[t] = np.vstack([Vt[a] @ Vs[:k], Vt[b] @ Vs[k:]])
    S = np.zeros((n, n))
    for t, nd_ in enumerate(nodes):
        if not nd_["children"]:
            R = slice(nd_["lo"], nd_["hi"])
            S[R, R] = rng.standard_normal((nd_["hi"] - nd_["lo"],) * 2)
        else:
            a, b = nd_["children"]
            Ra = slice(nodes[a]["lo"], nodes[a]["hi"])
            Rb = slice(nodes[b]["lo"], nodes[b]["hi"])
            S[Ra, Rb] = Ut[a] @ rng.standard_normal((k, k)) @ Vt[b].T
            S[Rb, Ra] = Ut[b] @ rng.standard_normal((k, k)) @ Vt[a].T
    return S


@pytest.mark.parametrize("n,leaf,k", [(128, 16, 4), (200, 24, 6), (96, 12, 3)])
def test_hss_recovers_hss_matrix(n, leaf, k):
    rng = np.random.default_rng(n)
    nodes = _nodes_binary(n, leaf)
    S = _hss_by_construction(nodes, k, rng)
    H, rep = hss_compress(S, nodes, 1e-12, seed=1, front_id=0)
    assert np.linalg.norm(H - S) <= 1e-9 * np.linalg.norm(S)
    assert max(rep["krow"].values()) <= k and max(rep["kcol"].values()) <= k
    assert rep["rounds"] == 1


def test_hss_tolerance_on_smooth_kernel():
    """Off-diagonal blocks of a smooth kernel are numerically low rank."""
    n = 256
    x = np.linspace(0, 1, n)
    S = 1.0 / (1.0 + 50.0 * np.abs(x[:, None] - x[None, :])) + np.eye(n)
    nodes = _nodes_binary(n, 32)
    for tol in (1e-4, 1e-8):
        H, rep = hss_compress(S, nodes, tol, seed=2, front_id=3)
        err = np.linalg.norm(H - S, 2) / np.linalg.norm(S, 2)
        depth = max(nd_["depth"] for nd_ in nodes)
        assert err <= 10 * tol * depth


def test_hss_adaptive_growth():
    """A rank above r - oversample forces a wider sample (r grows by 32)."""
    n = 256
    nodes = _nodes_binary(n, 64)
    rng = np.random.default_rng(4)
    S = _hss_by_construction(nodes, 30, rng)
    H, rep = hss_compress(S, nodes, 1e-12, seed=0, front_id=0)
    assert rep["r"] >= 64 and rep["rounds"] >= 2
    assert np.linalg.norm(H - S) <= 1e-8 * np.linalg.norm(S)


def test_single_node_is_identity():
    S = np.random.default_rng(0).standard_normal((20, 20))
    nodes = [dict(lo=0, hi=20, children=[], depth=0)]
    H, rep = hss_compress(S, nodes, 1e-4, 0, 0)
    assert np.array_equal(H, S)


def test_hss_capped_width_keeps_s():
    """Rank 30 needs r >= 40 samples (k + p, Theorem 1).  With the width
    capped at 32 the bound does not hold: the front keeps S exactly.  With
    room to grow (cap 64), the same matrix is recovered by the HSS build."""
    n = 256
    nodes = _nodes_binary(n, 64)
    S = _hss_by_construction(nodes, 30, np.random.default_rng(4))
    H, rep = hss_compress(S, nodes, 1e-12, seed=0, front_id=0, rmax=32)
    assert rep["capped"] and rep["r"] == 32 and rep["rounds"] == 1
    assert np.array_equal(H, S)
    H2, rep2 = hss_compress(S, nodes, 1e-12, seed=0, front_id=0, rmax=64)
    assert not rep2["capped"] and rep2["r"] == 64
    assert not np.array_equal(H2, S) and np.linalg.norm(H2 - S) <= 1e-8 * np.linalg.norm(S)
    # a low-rank matrix never reaches the cap
    S3 = _hss_by_construction(nodes, 4, np.random.default_rng(5))
    H3, rep3 = hss_compress(S3, nodes, 1e-12, seed=0, front_id=0, rmax=32)
    assert not rep3["capped"] and np.linalg.norm(H3 - S3) <= 1e-9 * np.linalg.norm(S3)
