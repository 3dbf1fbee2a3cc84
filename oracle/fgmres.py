"""Restarted flexible GMRES with right preconditioning.

The paper measures the preconditioner by GMRES iterations (Sec. 5) without
fixing the variant.  Reading used here: right-preconditioned flexible GMRES(m)
(Saad 1993), modified Gram-Schmidt Arnoldi, Givens rotations on the
Hessenberg matrix, x0 = 0 unless given.  A cycle stops when the Arnoldi
residual estimate |g_{j+1}| / ||b|| <= rtol; the method stops when the true
residual ||b - A x|| / ||b||, recomputed in FP64 at every restart, is <= rtol.
"""
import numpy as np


def fgmres(matvec, precond, b, x0=None, restart=30, rtol=1e-8, maxit=1000):
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, dict(iters=0, hist=[0.0], relres=0.0, converged=True)
    m = restart
    its = 0
    hist = []
    true_hist = []
    while True:
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        true_hist.append(rel)
        if rel <= rtol:
            return x, dict(iters=its, hist=hist, true_hist=true_hist, relres=rel, converged=True)
        if its >= maxit:
            return x, dict(iters=its, hist=hist, true_hist=true_hist, relres=rel, converged=False)
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        Hm = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        jend = 0
        for j in range(m):
            Z[:, j] = precond(V[:, j]) if precond is not None else V[:, j]
            w = matvec(Z[:, j])
            for i in range(j + 1):
                Hm[i, j] = float(w @ V[:, i])
                w = w - Hm[i, j] * V[:, i]
            hn = float(np.linalg.norm(w))
            Hm[j + 1, j] = hn
            if hn > 0.0:
                V[:, j + 1] = w / hn
            for i in range(j):
                a, c = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a + sn[i] * c
                Hm[i + 1, j] = -sn[i] * a + cs[i] * c
            a, c = Hm[j, j], Hm[j + 1, j]
            rr = float(np.hypot(a, c))
            cs[j], sn[j] = (a / rr, c / rr) if rr > 0.0 else (1.0, 0.0)
            Hm[j, j] = rr
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            jend = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= rtol or its >= maxit or hn == 0.0:
                break
        y = np.zeros(jend)
        for i in range(jend - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:jend] @ y[i + 1:jend]) / Hm[i, i]
        x = x + Z[:, :jend] @ y
