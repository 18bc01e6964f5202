"""Philox4x32-10 counter-based generator (NumPy, vectorised).

Published definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11 (2011), section 3.
A 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1) go through ten
rounds of

    (hi0, lo0) = mulhilo(M0, c0);  (hi1, lo1) = mulhilo(M1, c2)
    c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)

with the key bumped by the Weyl constants between rounds.  The CUDA twin in
``paper_2602_02500_gb300/csrc/synth.cu`` implements the same definition, so a
matrix generated on the device can be regenerated here bit for bit.

This module holds no arithmetic of the orthogonalisation method; it only turns
counters into integers and integers into exactly representable values.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Return the four 32-bit output words (uint32 arrays) for the counters.

    c0..c3 are broadcastable integer arrays (taken modulo 2^32); k0, k1 are
    python ints (the key is the same for every counter of one call).
    """
    shape = np.broadcast(np.asarray(c0), np.asarray(c1), np.asarray(c2), np.asarray(c3)).shape
    x0 = np.broadcast_to(np.asarray(c0, dtype=np.uint64) & MASK32, shape).copy()
    x1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64) & MASK32, shape).copy()
    x2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64) & MASK32, shape).copy()
    x3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64) & MASK32, shape).copy()
    ka = int(k0) & 0xFFFFFFFF
    kb = int(k1) & 0xFFFFFFFF
    for r in range(10):
        p0 = M0 * x0
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(ka)), lo1, (hi0 ^ x3 ^ np.uint64(kb)), lo0
        if r != 9:
            ka = (ka + W0) & 0xFFFFFFFF
            kb = (kb + W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def uniform53(words_hi, words_lo) -> np.ndarray:
    """Exact FP64 uniform in (0, 1) from two 32-bit words: 53 random bits + 1/2 ulp.

    u = ((hi >> 5) * 2^26 + (lo >> 6) + 0.5) * 2^-53, every step exact in FP64.
    """
    a = (np.asarray(words_hi, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(words_lo, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def uniform24(words) -> np.ndarray:
    """Exact FP32-representable uniform in (0, 1): ((w >> 8) + 0.5) * 2^-24."""
    a = (np.asarray(words, dtype=np.uint64) >> np.uint64(8)).astype(np.float64)
    return (a + 0.5) * (1.0 / 16777216.0)
