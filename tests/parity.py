"""Error measures of the parity tests (GPU result a against the oracle's b).

rel_fro  ||a - b||_F / ||b||_F                      (norm-wise)
rel_max  max|a - b| / max|b|                          (element-wise, on the scale of the whole matrix)
rel_col  max over columns j of max_i|a_ij - b_ij| / max_i|b_ij|   (each column on its own scale)
"""
import numpy as np


def rel_fro(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_col(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    a, b = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    den = np.maximum(np.abs(b).max(axis=0), 1e-300)
    return float((np.abs(a - b).max(axis=0) / den).max())
