"""Counter-based Rademacher (+-1) test matrices for randomized sampling.

Theorem 1 of the paper (Sec. 2) draws random test matrices (the T_rand term);
the paper fixes no distribution.  Reading used here: entries are +-1 with equal
probability, drawn from the SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA
2014; the constants are those of the published generator) applied to a
counter.  Entry (row, col) of stream s for front f under seed q is

    key  = q XOR (s << 62) XOR (f << 40) XOR (row << 20) XOR col
    sign = -1 if bit 63 of splitmix64(key) is set, else +1.

Columns are prefixes of one infinite stream, so growing the sample width keeps
earlier columns.  Limits: row, col < 2^20, f < 2^22, s < 4.
Streams: 0 = Omega (right samples), 1 = Psi (left samples), 2 = probes.
"""
import numpy as np

_C0 = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _C0
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher(seed: int, stream: int, front_id: int, rows, cols) -> np.ndarray:
    """float64 matrix of +-1, shape (len(rows), len(cols))."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.asarray(cols, dtype=np.uint64)
    base = (np.uint64(seed) ^ (np.uint64(stream) << np.uint64(62))
            ^ (np.uint64(front_id) << np.uint64(40)))
    key = base ^ (rows[:, None] << np.uint64(20)) ^ cols[None, :]
    h = splitmix64(key)
    neg = (h >> np.uint64(63)).astype(bool)
    return np.where(neg, -1.0, 1.0)
