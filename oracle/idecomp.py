"""Interpolative decomposition (paper Sec. 2, eq. (43) and its footnote).

An ID of an m x r matrix M by rows writes M ~= U M(J, :), where J holds k
selected ("skeleton") rows and U (m x k) contains the identity on the rows J.
The paper asks that no entry of the interpolation matrix exceed 2 in absolute
value (footnote on "well-behaved").

Steps (the textbook construction the paper cites, Cheng/Gimbutas/Martinsson/
Rokhlin style, written out):
  1. column-pivoted Householder QR of A = M^t (r x m): at step j the column of
     largest remaining norm is moved to position j (ties: lowest index);
  2. rank: k = the first j with |R_jj| <= tol * |R_11| (relative tolerance per
     ID; k = 0 for a zero matrix);
  3. T = argmin ||A(:,J) T - A(:,J^c)|| (= R11^-1 R12), the interpolation
     coefficients of the non-skeleton columns;
  4. while max |T_ij| > 2: exchange skeleton i with non-skeleton j at the
     largest entry (first in row-major order on ties) and recompute T (the
     Gu-Eisenstat exchange; each exchange grows |det R11| by more than 2, so
     the loop ends);
  5. U = Pi [I_k ; T^t].
"""
import numpy as np


def interp_decomp(M: np.ndarray, tol: float, max_swaps: int = 64):
    """Row ID of M (m x r).  Returns (U, J, T, info): U m x k, J skeleton row
    indices in selection order, T k x (m-k), info = {'k', 'swaps', 'order'}
    where order is the final column permutation [J, J^c]."""
    M = np.asarray(M, dtype=np.float64)
    m, r = M.shape
    A = M.T.copy()                  # r x m, one column per row of M
    R = A.copy()
    order = np.arange(m)
    kmax = min(r, m)
    k = 0
    first = 0.0
    for j in range(kmax):
        norms = np.sum(R[j:, j:] ** 2, axis=0)
        t = int(np.argmax(norms))
        nrm = float(np.sqrt(norms[t]))
        if j == 0:
            first = nrm
        if first == 0.0 or nrm <= tol * first:
            break
        piv = j + t
        if piv != j:
            R[:, [j, piv]] = R[:, [piv, j]]
            order[[j, piv]] = order[[piv, j]]
        # Householder reflector for R[j:, j]
        x = R[j:, j].copy()
        alpha = -np.copysign(np.linalg.norm(x), x[0]) if x[0] != 0 else -np.linalg.norm(x)
        v = x.copy()
        v[0] -= alpha
        vn = float(v @ v)
        if vn > 0.0:
            R[j:, j:] -= np.outer(v, (2.0 / vn) * (v @ R[j:, j:]))
        R[j + 1:, j] = 0.0
        k = j + 1

    J = order[:k].copy()
    Jc = order[k:].copy()
    T = _coeffs(A, J, Jc)
    swaps = 0
    while k > 0 and Jc.size > 0 and swaps < max_swaps:
        flat = int(np.argmax(np.abs(T)))
        i, jj = divmod(flat, T.shape[1])
        if abs(T[i, jj]) <= 2.0:
            break
        J[i], Jc[jj] = Jc[jj], J[i]
        T = _coeffs(A, J, Jc)
        swaps += 1
    U = np.zeros((m, k))
    U[J, np.arange(k)] = 1.0
    if Jc.size:
        U[Jc, :] = T.T
    return U, J, T, dict(k=k, swaps=swaps, order=np.concatenate([J, Jc]))


def _coeffs(A, J, Jc):
    """Least-squares interpolation coefficients T with A(:,J) T ~= A(:,J^c)."""
    if J.size == 0 or Jc.size == 0:
        return np.zeros((J.size, Jc.size))
    T, *_ = np.linalg.lstsq(A[:, J], A[:, Jc], rcond=None)
    return T
