"""Structured merge (reading R2): the approximate inverse of the interior block
of a parent front by the block solve of eq. (37), with the second diagonal
block compressed as in Theorem 1 (Algorithm 1 for a front, Algorithm 3 for
the top block A^(0)).

For a parent sigma with children mu, nu, the interior block of the front is

    A_ii = [[S^mu_ii, A^(mu,nu)], [A^(nu,mu), S^nu_ii]]

with S^mu_ii the restriction of the child approximant H^mu to B^mu n I^sigma
(Algorithm 1 step 2.1), and likewise for nu.  Step 2.2 compresses

    S~^nu_ii = S^nu_ii - A^(nu,mu) (S^mu_ii)^-1 A^(mu,nu)

to its HSS approximant H~ (Theorem 1, the same randomized construction and
options as the Schur complements), and eq. (37) applies

    x2 = H~^-1 (z2 - A^(nu,mu) (S^mu_ii)^-1 z1)
    x1 = (S^mu_ii)^-1 z1 - (S^mu_ii)^-1 A^(mu,nu) x2.

The fast HSS inversions of the paper are exact up to rounding; this oracle
forms the same inverses densely, so it computes what R2 computes without its
complexity.  Written out as a matrix, the block solve is the exact inverse of
A_ii + blockdiag(0, H~ - S~) (a test checks this identity).

Readings where the paper is silent: the HSS tree of S~^nu_ii is the
nested-dissection subtree of nu restricted to B^nu n I^sigma (the tree rule
of the Schur complements, c3); its random test matrices use the counter key
nbox + sigma (nbox + nbox for the top block), so they are independent of the
Schur complements' own; tolerance, widths, oversampling, cap policy and probe
are those of the Schur complements.

This is test infrastructure, like the rest of the package.
"""
import numpy as np

from .hss import hss_compress


def block_inverse(Aii, n1, nodes, tol, seed, key, **kw):
    """The dense matrix of eq. (37)'s block solve for Aii = [[S1, A12], [A21,
    S2]] (S1 of size n1), with S~2 = S2 - A21 S1^-1 A12 replaced by its HSS
    approximant over `nodes` (None: not compressed).  Returns (X, info) with
    info holding S~2, its approximant H~ and the compression report."""
    n = Aii.shape[0]
    S1, A12 = Aii[:n1, :n1], Aii[:n1, n1:]
    A21, S2 = Aii[n1:, :n1], Aii[n1:, n1:]
    S1inv = np.linalg.inv(S1) if n1 else np.zeros((0, 0))
    St = S2 - A21 @ S1inv @ A12
    if nodes is not None and St.shape[0] > 0 and len(nodes) > 1:
        Ht, rep = hss_compress(St, nodes, tol, seed, key, **kw)
    else:
        Ht, rep = St.copy(), None
    Htinv = np.linalg.inv(Ht) if Ht.shape[0] else np.zeros((0, 0))
    X = np.zeros((n, n))
    G = S1inv @ A12                          # S1^-1 A12
    E = A21 @ S1inv                          # A21 S1^-1
    X[:n1, :n1] = S1inv + G @ Htinv @ E
    X[:n1, n1:] = -G @ Htinv
    X[n1:, :n1] = -Htinv @ E
    X[n1:, n1:] = Htinv
    return X, dict(St=St, Ht=Ht, rep=rep)


def interior_split(nd, b):
    """Number of interior dofs of the parent front of box b that come from
    its first child (B^mu n I^b leads the interior set, then B^nu n I^b), and
    the second child's dofs in that set (in their stored order)."""
    ni = nd["iset"][b].size
    mu, nu = (int(c) for c in nd["child"][b])
    fm, fn = nd["fmap"][mu], nd["fmap"][nu]
    pm, pn = np.sort(fm[fm < ni]), np.sort(fn[fn < ni])
    n1 = pm.size
    assert np.array_equal(pm, np.arange(n1)) and np.array_equal(pn, np.arange(n1, ni))
    return n1, nd["bset"][nu][fn < ni]
