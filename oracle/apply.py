"""Application of the inverse factorization M^-t D^-1 L^-1 (end of Sec. 4.2).

With the Gauss transforms of Sec. 4.1, L(B,I) = F_bi F_ii^-1 and
M(B,I)^t = F_ii^-1 F_ib = W, solving L D M^t y = x box by box is:
  forward, in elimination order:  t_sigma = F_ii^-1 x_I ;  x_B -= F_bi t_sigma
  top:                            x_top = A^(0)^-1 x_top           (eq. (36))
  backward, reverse order:        x_I = t_sigma - W x_B
Under the structured merge (reading R2) F_ii^-1 and A^(0)^-1 are the
approximate inverses of eq. (37) (Algorithms 1 and 3), stored densely.
Vectors are in the original dof numbering; x may have several columns.
"""
import numpy as np
import scipy.linalg as sla


def apply(fac, x):
    nd = fac["nd"]
    w = np.array(x, dtype=np.float64, copy=True)
    squeeze = w.ndim == 1
    if squeeze:
        w = w[:, None]
    t = {}
    for b in nd["order"]:
        b = int(b)
        I, B = nd["iset"][b], nd["bset"][b]
        f = fac["boxes"][b]
        if I.size == 0:
            continue
        tb = f["Xinv"] @ w[I] if f.get("Xinv") is not None else sla.lu_solve(f["lu"], w[I])
        w[B] -= f["Fbi"] @ tb
        t[b] = tb
    top = fac["top"]
    if top.size:
        if fac.get("top_inv") is not None:
            w[top] = fac["top_inv"] @ w[top]
        else:
            w[top] = sla.lu_solve(fac["top_lu"], w[top])
    for b in nd["order"][::-1]:
        b = int(b)
        I, B = nd["iset"][b], nd["bset"][b]
        if I.size == 0:
            continue
        w[I] = t[b] - fac["boxes"][b]["W"] @ w[B]
    return w[:, 0] if squeeze else w
