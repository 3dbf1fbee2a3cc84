"""Randomized HSS approximation of a Schur complement (paper Sec. 2, Theorem 1).

Theorem 1 (the construction of Martinsson, SIMAX 2011, that the paper cites)
builds an HSS representation from 2(k+p) products with the matrix and its
transpose plus O(Nk) matrix entries, compressing the off-diagonal blocks by
interpolative decompositions with nested bases (Sec. 2: U^tall_sigma =
diag(U^tall_mu, U^tall_nu) U_sigma, and the same for V).

Steps, bottom-up over the HSS tree (leaves first):
  * samples Y = S Omega, Z = S^t Psi with +-1 test matrices of width r;
  * leaf tau with index range R: local samples Y_tau = Y(R,:) - S(R,R) Omega(R,:),
    Z_tau = Z(R,:) - S(R,R)^t Psi(R,:);
  * parent tau of the sibling pair (a, b):
        Y_tau = [Y_a(J_a,:) ; Y_b(J_b,:)] - [0 B_ab ; B_ba 0] [Om_a ; Om_b],
        Z_tau = [Z_a(K_a,:) ; Z_b(K_b,:)] - [0 B_ba^t ; B_ab^t 0] [Ps_a ; Ps_b],
    with B_ab = S(J_a, K_b) and the compressed test matrices
    Om_tau = V_tau^t Omega_local, Ps_tau = U_tau^t Psi_local;
  * row ID of Y_tau gives U_tau and skeleton rows J_tau (S row indices);
    row ID of Z_tau gives V_tau and skeleton columns K_tau;
  * leaves keep D_tau = S(R,R); sibling pairs keep B_ab = S(J_a, K_b).

Readings where the paper is silent:
  * the HSS tree of S^sigma is the nested-dissection subtree of sigma restricted
    to B^sigma, with empty boxes removed and single-child chains collapsed;
  * oversampling p = 10 (Theorem 1's typical value); the sample width r starts
    at 32 and grows by 32 (whole front redone, earlier columns kept) while some
    node's rank exceeds r - 10 and r < n (and, when a cap rmax is given, while
    r + 32 <= rmax);
  * the ID tolerance is relative per ID (see idecomp.py);
  * when the cap rmax stops the growth while some rank still exceeds r - 10,
    Theorem 1's error bound (which needs k + p samples) does not apply, and
    the front keeps S itself (H = S, rep["capped"] = True) under the default
    cap policy "keep"; under the policy "accept" it keeps the approximant
    built from the r samples it has (ranks up to r, no error bound), which is
    the fixed anticipated rank l of the paper's experiments (Sec. 5: l chosen
    beforehand, the preconditioner judged by the GMRES iterations).
  * residual probe (optional, the fallback check of the learned-width form):
    an approximant accepted by the rank test above is checked on nprobe +-1
    vectors W from stream 2, ||(S - H) W||_F / ||S W||_F <= 10 tol depth (the
    HSS tree depth, at least 1); a front that fails samples again with r + 32
    while the cap allows, like a front short of samples.  On adaptive runs at
    tol 1e-4 and 1e-6 the largest ratio to tol depth seen was 1.2.
The approximant is returned expanded to a dense matrix H (the parent front is
built from H, eq. (32)), together with the representation and its ranks.
"""
import numpy as np

from .idecomp import interp_decomp
from .rademacher import rademacher


def hss_tree_for_front(nd, box, dofs=None):
    """HSS tree over the index set B^box (in its stored order), or over a
    subset `dofs` of it (kept in that order; the structured merge compresses
    blocks indexed by B^box n I^parent).

    Returns a list of nodes; each node is a dict with 'lo', 'hi' (range inside
    the index set), 'children' (node indices) and 'depth'.  The last node is
    the root.
    """
    bs_dofs = nd["bset"][box] if dofs is None else np.asarray(dofs)
    if bs_dofs.size == 0:
        return []
    dfs_pos = np.empty(nd["dfs_dof"].size, dtype=np.int64)
    dfs_pos[nd["dfs_dof"]] = np.arange(nd["dfs_dof"].size)
    pos = dfs_pos[bs_dofs]                 # ascending (B^box is DFS ordered)
    child = nd["child"]
    nodes = []

    def build(b):
        lo = int(np.searchsorted(pos, nd["pos0"][b], side="left"))
        hi = int(np.searchsorted(pos, nd["pos1"][b], side="left"))
        if hi == lo:
            return None
        if child[b, 0] < 0:
            nodes.append(dict(lo=lo, hi=hi, children=[]))
            return len(nodes) - 1
        c0 = build(child[b, 0])
        c1 = build(child[b, 1])
        if c0 is None:
            return c1
        if c1 is None:
            return c0
        nodes.append(dict(lo=lo, hi=hi, children=[c0, c1]))
        return len(nodes) - 1

    root = build(box)
    assert root == len(nodes) - 1
    # depth from the root
    nodes[root]["depth"] = 0
    for i in range(len(nodes) - 1, -1, -1):
        for c in nodes[i]["children"]:
            nodes[c]["depth"] = nodes[i]["depth"] + 1
    return nodes


def hss_compress(S, nodes, tol, seed, front_id, r0=32, dr=32, oversample=10, rmax=None, cap="keep", probe=0):
    """Randomized HSS approximant of S.  Returns (H, rep) with H dense.

    rmax (optional) caps the sample width: growth stops once r + dr > rmax,
    and a front whose ranks still need more samples then returns H = S
    (cap="keep") or the approximant from the r samples (cap="accept").
    probe > 0: residual probe of an accepted approximant (see module notes)."""
    if cap not in ("keep", "accept"):
        raise ValueError("cap policy: 'keep' or 'accept'")
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    root = len(nodes) - 1
    if n == 0 or len(nodes) == 1:
        return S.copy(), dict(r=0, rounds=0, krow={}, kcol={}, nodes=nodes, swaps=0)
    # process order: deeper nodes first (children before parents)
    order = sorted(range(root), key=lambda i: (-nodes[i]["depth"], i))
    r = r0 if rmax is None else min(r0, rmax)
    rounds = 0
    probe_regrown = 0
    probe_rel = None
    while True:
        rounds += 1
        Om = rademacher(seed, 0, front_id, np.arange(n), np.arange(r))
        Ps = rademacher(seed, 1, front_id, np.arange(n), np.arange(r))
        Y = S @ Om
        Z = S.T @ Ps
        st = {}
        for t in order:
            nd_ = nodes[t]
            if not nd_["children"]:
                R = np.arange(nd_["lo"], nd_["hi"])
                Yl = Y[R] - S[np.ix_(R, R)] @ Om[R]
                Zl = Z[R] - S[np.ix_(R, R)].T @ Ps[R]
                rows, cols = R, R
                Oml, Psl = Om[R], Ps[R]
            else:
                a, b = nd_["children"]
                A_, B_ = st[a], st[b]
                Bab = S[np.ix_(A_["J"], B_["K"])]
                Bba = S[np.ix_(B_["J"], A_["K"])]
                Yl = np.vstack([A_["Yskel"] - Bab @ B_["Omt"], B_["Yskel"] - Bba @ A_["Omt"]])
                Zl = np.vstack([A_["Zskel"] - Bba.T @ B_["Pst"], B_["Zskel"] - Bab.T @ A_["Pst"]])
                rows = np.concatenate([A_["J"], B_["J"]])
                cols = np.concatenate([A_["K"], B_["K"]])
                Oml = np.vstack([A_["Omt"], B_["Omt"]])
                Psl = np.vstack([A_["Pst"], B_["Pst"]])
            U, Jl, _, iu = interp_decomp(Yl, tol)
            V, Kl, _, iv = interp_decomp(Zl, tol)
            st[t] = dict(U=U, V=V, J=rows[Jl], K=cols[Kl], Yskel=Yl[Jl], Zskel=Zl[Kl],
                         Omt=V.T @ Oml, Pst=U.T @ Psl, swaps=iu["swaps"] + iv["swaps"])
        kmax = max(max(st[t]["U"].shape[1], st[t]["V"].shape[1]) for t in order)
        short_of_samples = kmax > r - oversample and r < n
        if short_of_samples and (rmax is None or r + dr <= rmax):
            r += dr
            continue
        if probe > 0 and not short_of_samples:
            H = _expand(S, nodes, st, order)
            probe_rel = probe_residual(S, H, seed, front_id, probe)
            if probe_rel > probe_threshold(tol, nodes) and (rmax is None or r + dr <= rmax) and r < n:
                r += dr
                probe_regrown += 1
                continue
        break
    if short_of_samples and cap == "keep":
        return S.copy(), dict(r=r, rounds=rounds, nodes=nodes, capped=True,
                              krow={t: st[t]["U"].shape[1] for t in order},
                              kcol={t: st[t]["V"].shape[1] for t in order},
                              swaps=sum(st[t]["swaps"] for t in order))

    H = _expand(S, nodes, st, order)
    rep = dict(r=r, rounds=rounds, nodes=nodes, capped=bool(short_of_samples), truncated=bool(short_of_samples),
               probe_rel=probe_rel, probe_regrown=probe_regrown,
               krow={t: st[t]["U"].shape[1] for t in order},
               kcol={t: st[t]["V"].shape[1] for t in order},
               J={t: st[t]["J"] for t in order}, K={t: st[t]["K"] for t in order},
               U={t: st[t]["U"] for t in order}, V={t: st[t]["V"] for t in order},
               swaps=sum(st[t]["swaps"] for t in order))
    return H, rep


def _expand(S, nodes, st, order):
    """Dense H from the representation: U^tall / V^tall bottom-up (nested
    bases), leaf diagonal blocks D = S(R, R), sibling blocks
    U^tall_a S(J_a, K_b) V^tall_b^t."""
    Ut, Vt = {}, {}
    for t in order:
        ch = nodes[t]["children"]
        if not ch:
            Ut[t], Vt[t] = st[t]["U"], st[t]["V"]
        else:
            a, b = ch
            Ut[t] = _blkdiag(Ut[a], Ut[b]) @ st[t]["U"]
            Vt[t] = _blkdiag(Vt[a], Vt[b]) @ st[t]["V"]
    H = np.zeros_like(S)
    for t in range(len(nodes)):
        nd_ = nodes[t]
        if not nd_["children"]:
            R = slice(nd_["lo"], nd_["hi"])
            H[R, R] = S[R, R]
        else:
            a, b = nd_["children"]
            Ra = slice(nodes[a]["lo"], nodes[a]["hi"])
            Rb = slice(nodes[b]["lo"], nodes[b]["hi"])
            H[Ra, Rb] = Ut[a] @ S[np.ix_(st[a]["J"], st[b]["K"])] @ Vt[b].T
            H[Rb, Ra] = Ut[b] @ S[np.ix_(st[b]["J"], st[a]["K"])] @ Vt[a].T
    return H


def probe_residual(S, H, seed, front_id, nprobe):
    """||(S - H) W||_F / ||S W||_F for nprobe +-1 probe vectors W (stream 2 of
    the counter generator); 0 when S W = 0."""
    W = rademacher(seed, 2, front_id, np.arange(S.shape[0]), np.arange(nprobe))
    den = np.linalg.norm(S @ W)
    return float(np.linalg.norm((S - H) @ W) / den) if den > 0 else 0.0


def probe_threshold(tol, nodes):
    """10 tol times the depth of the HSS tree (at least 1): the errors of the
    nested IDs along a root-to-leaf path add up."""
    return 10.0 * tol * max(1, max(nd_["depth"] for nd_ in nodes))


def _blkdiag(X, Y):
    out = np.zeros((X.shape[0] + Y.shape[0], X.shape[1] + Y.shape[1]))
    out[: X.shape[0], : X.shape[1]] = X
    out[X.shape[0]:, X.shape[1]:] = Y
    return out
