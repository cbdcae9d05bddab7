"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4x32-bit counter and a 2x32-bit key; each of the ten rounds
multiplies counter words 0 and 2 by two fixed odd constants, keeps the 64-bit
products' high and low halves, mixes the high halves with the other two words
and the key, and the key is advanced by two Weyl constants between rounds.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. All arguments are array-likes of 32-bit
    values (broadcast together); returns four uint64 arrays holding the
    32-bit output words."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    for _ in range(10):
        p0 = _M0 * c0  # < 2^64: exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def trajectory_uniforms(seed: int, b_index: int, s: np.ndarray, k: int) -> np.ndarray:
    """32-bit uniform words u_j for gates j = 0..k-1 of trajectories ``s`` of
    bitstring ``b_index``: word (j mod 4) of the Philox block with counter
    (floor(j/4), s, b_index low word, b_index high word) and key
    (seed low word, seed high word). Returns uint64 array of shape (len(s), k)."""
    s = np.asarray(s, dtype=np.uint64).reshape(-1, 1)
    nblk = (k + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64).reshape(1, -1)
    b_lo = np.uint64(b_index & 0xFFFFFFFF)
    b_hi = np.uint64((b_index >> 32) & 0xFFFFFFFF)
    s_lo = np.uint64(seed & 0xFFFFFFFF)
    s_hi = np.uint64((seed >> 32) & 0xFFFFFFFF)
    w0, w1, w2, w3 = philox4x32_10(blk, s, b_lo, b_hi, s_lo, s_hi)
    words = np.stack([w0, w1, w2, w3], axis=-1).reshape(s.shape[0], nblk * 4)
    return words[:, :k]
