"""Block ILU(0) of a BSR matrix: the incomplete factorization that the paper
compares its preconditioner with (Sec. 5, "a standard ILU preconditioner").

ILU(0) keeps exactly the block sparsity of A.  L is block unit lower
triangular on A's strictly lower pattern, U is block upper triangular on A's
upper pattern (diagonal included), and the product L U equals A at every
block position of A's pattern; fill outside the pattern is dropped.  The
elimination runs in the natural order of the block rows (elements), as
Gaussian elimination in row form, block by block:

  for each block row i, for each k < i in row i's pattern, ascending:
      A_ik <- A_ik U_kk^-1
      for each j > k in row k's pattern that is also in row i's pattern:
          A_ij <- A_ij - A_ik U_kj
  then L_ik = A_ik (k < i), U_ij = A_ij (j >= i).

The preconditioner is z = U^-1 L^-1 x, by forward then backward block
substitution.

Readings where the paper is silent: it names "a standard ILU preconditioner"
without its variant.  Zero fill on the block pattern of A is used, in the
natural element order, with right preconditioning inside the same FGMRES.
Since every stored block of A is dense, the block form equals scalar ILU(0)
on A's scalar pattern (a test checks this on small meshes).

This is test infrastructure, like the rest of the package.
"""
import numpy as np


def ilu0(row_ptr, col_idx, val):
    """Block ILU(0).  row_ptr/col_idx: BSR structure (block columns ascending
    per row), val: (nnzb, bs, bs) blocks.  Returns a dict holding the factored
    blocks (L strictly below the diagonal, U on and above it) in A's layout."""
    row_ptr = np.asarray(row_ptr)
    col_idx = np.asarray(col_idx)
    F = np.array(val, dtype=np.float64, copy=True)
    nb = row_ptr.size - 1
    pos = [dict((int(col_idx[q]), q) for q in range(row_ptr[i], row_ptr[i + 1])) for i in range(nb)]
    for i in range(nb):
        for k in sorted(c for c in pos[i] if c < i):
            qik = pos[i][k]
            F[qik] = np.linalg.solve(F[pos[k][k]].T, F[qik].T).T      # A_ik U_kk^-1
            for j, qkj in pos[k].items():
                if j > k and j in pos[i]:
                    F[pos[i][j]] -= F[qik] @ F[qkj]
    return dict(row_ptr=row_ptr, col_idx=col_idx, F=F, pos=pos, nb=nb, bs=F.shape[1])


def ilu0_apply(ilu, x):
    """z = U^-1 L^-1 x (x: N or N x nrhs, N = nb * bs, block-row order)."""
    nb, bs, F, pos = ilu["nb"], ilu["bs"], ilu["F"], ilu["pos"]
    w = np.array(x, dtype=np.float64, copy=True)
    squeeze = w.ndim == 1
    if squeeze:
        w = w[:, None]
    w = w.reshape(nb, bs, -1)
    for i in range(nb):                        # L y = x (unit diagonal)
        for k, q in pos[i].items():
            if k < i:
                w[i] -= F[q] @ w[k]
    for i in range(nb - 1, -1, -1):            # U z = y
        for j, q in pos[i].items():
            if j > i:
                w[i] -= F[q] @ w[j]
        w[i] = np.linalg.solve(F[pos[i][i]], w[i])
    w = w.reshape(nb * bs, -1)
    return w[:, 0] if squeeze else w


def ilu0_dense_factors(ilu):
    """Dense L (unit lower) and U of a block ILU(0), for checks on small cases."""
    nb, bs, F, pos = ilu["nb"], ilu["bs"], ilu["F"], ilu["pos"]
    N = nb * bs
    L, U = np.eye(N), np.zeros((N, N))
    for i in range(nb):
        for j, q in pos[i].items():
            blk = (slice(i * bs, (i + 1) * bs), slice(j * bs, (j + 1) * bs))
            if j < i:
                L[blk] = F[q]
            else:
                U[blk] = F[q]
    return L, U
