"""Learned sample widths: training data from the method's own adaptive runs,
and per-box initial widths from a trained model (argument marshalling over
the C ABI; the features, the network and the factorization run in the
library).

A training sample is one compressed front of an adaptive factorization: its
six box features (hssnd.rank_features) and the target log(1 + k), k the
largest HSS node rank the adaptive ID found for it.
"""
from __future__ import annotations

import numpy as np

from . import hssnd


def logged_ranks(tree: hssnd.Tree, factor: hssnd.Factor, feats: np.ndarray):
    """(X, t) of the compressed fronts of one factorization."""
    log = factor.export_log()
    keep = log["r"] > 0
    boxes = log["box"][keep]
    return feats[boxes].astype(np.float32), np.log1p(log["kmax"][keep].astype(np.float64)).astype(np.float32)


def training_set(problems, tol, precision="fp32", rmax=96, leaf_max=64):
    """problems: iterable of (meshdesc, BSR, c_elem or None, kappa_h).  Runs
    nd_order + the adaptive hss_factor on each and collects (X, t)."""
    Xs, ts = [], []
    for meshdesc, A, c_elem, kappa_h in problems:
        dA = hssnd.DeviceBSR.from_host(A)
        tree = hssnd.nd_order(meshdesc, dA, leaf_max=leaf_max)
        F = hssnd.hss_factor(dA, tree, tol=tol, precision=precision, rmax=rmax)
        X, t = logged_ranks(tree, F, hssnd.rank_features(tree, c_elem, kappa_h))
        Xs.append(X)
        ts.append(t)
    return np.concatenate(Xs), np.concatenate(ts)


def widths(model: hssnd.RankModel, feats: np.ndarray, oversample=10, rmax=96) -> np.ndarray:
    """Initial sample width of every box (int32, HOST) from BF16 inference."""
    _, r = model.predict(feats, oversample=oversample, rmax=rmax)
    return r.astype(np.int32)
