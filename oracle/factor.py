"""Approximate LDM^t factorization over the box tree (paper Algorithm 2).

Reading R1 (the one this oracle implements): every Schur complement is
replaced by its HSS approximant H (Algorithm 2, steps 1 and 2), the parent
front is assembled from the children's H and the original coupling blocks
(eq. (32)), its interior block is factored densely, and the top block
A^(0) = [[H^1, A^(1,2)], [A^(2,1), H^2]] (eq. (36)) is factored densely.

Per box sigma, with front index set [I ; B] (I = I^sigma at leaves, I^ above):
  F      = A(front, front) at a leaf; above, F(i,j) = H^mu(i,j) when i,j lie in
           B^mu, H^nu(i,j) when i,j lie in B^nu, and A(i,j) otherwise (eq. (32));
  W      = F_ii^-1 F_ib                (M^(sigma)(B,I)^t, Sec. 4.1)
  S      = F_bb - F_bi W               (eq. (32))
  H      = HSS approximant of S        (Theorem 1), or S when compression is off.
Stored for the apply: the LU factors of F_ii, F_bi and W.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .hss import hss_tree_for_front, hss_compress
from .merge import block_inverse, interior_split


def csr_from_bsr(nb, bs, row_ptr, col_idx, val):
    M = sp.bsr_matrix((np.asarray(val, dtype=np.float64).reshape(-1, bs, bs),
                       np.asarray(col_idx), np.asarray(row_ptr)), shape=(nb * bs, nb * bs))
    return M.tocsr()


def box_schur(A_csr, nd, b):
    """Exact Schur complement of box b onto its boundary set B^b: the box's
    dofs are the I sets of its whole subtree plus B^b, and S = F_bb -
    F_bi F_ii^-1 F_ib with F = A(box, box) (Sec. 3, block elimination of the
    box interior).  It equals the S that Algorithm 2 forms at b whenever no
    Schur complement below b was approximated (compression off, or every
    descendant kept its S), so boxes of a large problem can be checked one
    at a time.  Rows and columns follow the stored order of B^b."""
    A = A_csr.tocsr()
    stack, inner = [int(b)], []
    while stack:
        c = stack.pop()
        inner.append(nd["iset"][c])
        if not nd["is_leaf"][c]:
            stack.extend(int(x) for x in nd["child"][c])
    I = np.concatenate(inner) if inner else np.zeros(0, dtype=np.int64)
    B = nd["bset"][b]
    idx = np.concatenate([I, B])
    F = A[idx][:, idx].toarray()
    ni = I.size
    if ni == 0:
        return F[ni:, ni:].copy()
    W = sla.lu_solve(sla.lu_factor(F[:ni, :ni]), F[:ni, ni:])
    return F[ni:, ni:] - F[ni:, :ni] @ W


def eliminate_front(F, ni):
    """Elimination of the interior block of one front (Sec. 4.1, eq. (32)):
    F = [F_ii F_ib; F_bi F_bb] with the first ni rows/columns interior;
    LU with partial pivoting of F_ii, W = F_ii^-1 F_ib (= M(B,I)^t) and the
    Schur complement S = F_bb - F_bi W.  Returns dict(lu, W, S); lu is None
    when ni = 0."""
    F = np.asarray(F, dtype=np.float64)
    Fii, Fib = F[:ni, :ni], F[:ni, ni:]
    Fbi, Fbb = F[ni:, :ni], F[ni:, ni:]
    if ni > 0:
        lu = sla.lu_factor(Fii)
        W = sla.lu_solve(lu, Fib)
    else:
        lu = None
        W = np.zeros((0, F.shape[0] - ni))
    return dict(lu=lu, W=W, S=Fbb - Fbi @ W)


def factor(A_csr, nd, tol=1e-6, seed=0, compress=True, r0=32, dr=32, oversample=10, rmax=None,
           keep_h=False, cap="keep", probe=0, r_init=None, merge="dense"):
    """Returns a dict with the per-box factors, the top block LU and logs.
    rmax caps the HSS sample width; cap is the policy for a front whose ranks
    outgrow the cap ("keep": H = S; "accept": the approximant from the samples
    it has, see hss.py); probe > 0 checks each accepted approximant on that
    many +-1 vectors and samples again when the check fails (hss.py);
    r_init (optional) maps a box id to its first sample width (the learned
    widths), in place of r0; keep_h stores each approximant H.
    merge="dense" is reading R1; merge="structured" is reading R2: each
    parent's interior block and the top block are inverted by the block solve
    of eq. (37) with the second Schur complement compressed (merge.py).  The
    apply then uses those approximate inverses (stored densely as "Xinv" and
    "top_inv")."""
    if cap not in ("keep", "accept"):
        raise ValueError("cap policy: 'keep' or 'accept'")
    if merge not in ("dense", "structured"):
        raise ValueError("merge: 'dense' or 'structured'")
    structured = merge == "structured" and compress
    ckw = dict(r0=r0, dr=dr, oversample=oversample, rmax=rmax, cap=cap, probe=probe)
    nbox = int(nd["nbox"])
    A = A_csr.tocsr()
    boxes = {}
    H = {}
    log = []
    for b in nd["order"]:
        b = int(b)
        I = nd["iset"][b]
        B = nd["bset"][b]
        ni = I.size
        if nd["is_leaf"][b]:
            idx = np.concatenate([I, B])
            F = A[idx][:, idx].toarray()
        else:
            mu, nu = (int(c) for c in nd["child"][b])
            idx = np.concatenate([I, B])
            F = A[idx][:, idx].toarray()
            for c in (mu, nu):
                fm = nd["fmap"][c]
                F[np.ix_(fm, fm)] = H.pop(c)
        Fii, Fib = F[:ni, :ni], F[:ni, ni:]
        Fbi, Fbb = F[ni:, :ni], F[ni:, ni:]
        rec = dict(box=b, level=int(nd["level"][b]), ni=ni, nb=B.size)
        Xinv = None
        if ni > 0 and structured and not nd["is_leaf"][b]:
            # Algorithm 1: block solve of eq. (37), S~ of the second child compressed
            n1, dofs2 = interior_split(nd, b)
            nodes2 = hss_tree_for_front(nd, int(nd["child"][b][1]), dofs2)
            Xinv, minfo = block_inverse(Fii, n1, nodes2, tol, seed, nbox + b, **ckw)
            rec["tilde"] = minfo
            lu = None
            W = Xinv @ Fib
        else:
            el = eliminate_front(F, ni)
            lu, W = el["lu"], el["W"]
        S = Fbb - Fbi @ W
        if compress and B.size > 0:
            nodes = hss_tree_for_front(nd, b)
            rb = r0 if r_init is None else max(1, min(int(r_init[b]), rmax if rmax is not None else 1 << 30))
            Hs, rep = hss_compress(S, nodes, tol, seed, b, r0=rb, dr=dr, oversample=oversample, rmax=rmax,
                                   cap=cap, probe=probe)
            rec.update(r=rep["r"], rounds=rep["rounds"], capped=rep.get("capped", False),
                       probe_regrown=rep.get("probe_regrown", 0), probe_rel=rep.get("probe_rel"),
                       kmax=max(list(rep["krow"].values()) + list(rep["kcol"].values()) + [0]),
                       nnodes=len(nodes), rep=rep)
        else:
            Hs = S.copy()
        H[b] = Hs
        boxes[b] = dict(lu=lu, Fbi=Fbi.copy(), W=W, S=S, F=F, Xinv=Xinv)
        if keep_h:
            boxes[b]["H"] = Hs.copy()
        log.append(rec)
    # top block, eq. (36)
    B0, B1 = nd["bset"][0], nd["bset"][1]
    top = np.concatenate([B0, B1])
    A0 = A[top][:, top].toarray()
    A0[np.ix_(nd["fmap"][0], nd["fmap"][0])] = H.pop(0)
    A0[np.ix_(nd["fmap"][1], nd["fmap"][1])] = H.pop(1)
    top_inv, top_info = None, None
    if structured and top.size:
        # Algorithm 3: S^1 = H^1 inverted, S~^2 = H^2 - A^(2,1) (H^1)^-1 A^(1,2) compressed
        top_inv, top_info = block_inverse(A0, B0.size, hss_tree_for_front(nd, 1), tol, seed, 2 * nbox, **ckw)
        top_lu = None
    else:
        top_lu = sla.lu_factor(A0) if top.size else None
    return dict(boxes=boxes, top=top, top_lu=top_lu, top_inv=top_inv, top_info=top_info, A0=A0, log=log, nd=nd,
                merge=merge)
