"""Counter-based Gaussian stream used for the random test matrices of the
randomized SVD (Sec. 3.1: Omega with i.i.d. Gaussian entries) and for the
random initial guess of the fit (Sec. 2.3.5).

ORACLE: test infrastructure only (tests/, smoke(), bench.py's CPU baseline).

Philox4x32-10 is written here from its published definition (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 10-round
bijection of a 128-bit counter under a 64-bit key; each round multiplies words
0 and 2 by fixed 32-bit constants, takes the high/low halves, and xors the high
halves with the other two words and the round key; the key advances by the
Weyl constants between rounds.

Gaussian mapping (the same definition is implemented independently on the
GPU): element ``i`` of stream ``s`` under ``seed`` uses counter
``(i mod 2^32, i >> 32, s mod 2^32, s >> 32)`` and key
``(seed mod 2^32, seed >> 32)``; with outputs ``x0..x3``,
``ua = (x0 * 2^21 + (x1 >> 11)) * 2^-53``, ``ub = (x2 * 2^21 + (x3 >> 11)) * 2^-53``,
and the value is ``sqrt(-2 ln(1 - ua)) * cos(2 pi ub)`` (Box-Muller).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def normals(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` Gaussian values of ``stream`` starting at element ``start``."""
    i = np.arange(start, start + count, dtype=np.uint64)
    seed = np.uint64(seed)
    stream = np.uint64(stream)
    x0, x1, x2, x3 = philox4x32_10(i & MASK, i >> np.uint64(32), stream & MASK,
                                   stream >> np.uint64(32), seed & MASK, seed >> np.uint64(32))
    two21 = np.uint64(1 << 21)
    ua = (x0 * two21 + (x1 >> np.uint64(11))).astype(np.float64) * 2.0 ** -53
    ub = (x2 * two21 + (x3 >> np.uint64(11))).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log1p(-ua)) * np.cos(2.0 * np.pi * ub)


# Stream identifiers (shared convention with the GPU side, restated there).
def omega_stream(sweep: int, site: int) -> int:
    """Stream of the sketch matrix of sweep ``sweep`` (0-based) at window ``site`` (1-based)."""
    return (1 << 40) | (sweep << 20) | site


def init_stream(site: int) -> int:
    """Stream of the Gaussian initial-guess core of site ``site`` (1-based)."""
    return (2 << 40) | site
