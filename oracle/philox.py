"""Philox4x32-10 counter-based generator (oracle; test infrastructure only).

Written from its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11): a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1);
each round multiplies c0 and c2 by fixed 32-bit multipliers, splits the 64-bit products into
high and low words and recombines them with c1, c3 and the key; the key is advanced by two
fixed Weyl increments between rounds; ten rounds.

Used only to check the library's generator bit for bit. The simulator's own random numbers in
the oracle come from numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

MULT_0 = 0xD2511F53
MULT_1 = 0xCD9E8D57
WEYL_0 = 0x9E3779B9
WEYL_1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _round(c, k):
    p0 = MULT_0 * c[0]
    p1 = MULT_1 * c[2]
    hi0, lo0 = (p0 >> 32) & MASK32, p0 & MASK32
    hi1, lo1 = (p1 >> 32) & MASK32, p1 & MASK32
    return [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]


def philox4x32_10(counter, key):
    """One block: counter = 4 uint32, key = 2 uint32 -> 4 uint32 (Python ints)."""
    c = [int(v) & MASK32 for v in counter]
    k = [int(v) & MASK32 for v in key]
    for r in range(10):
        if r > 0:
            k = [(k[0] + WEYL_0) & MASK32, (k[1] + WEYL_1) & MASK32]
        c = _round(c, k)
    return c


def philox_array(counters: np.ndarray, key) -> np.ndarray:
    """Vectorised form: counters [M, 4] uint32 -> [M, 4] uint32, same key for all."""
    c = [counters[:, i].astype(np.uint64) for i in range(4)]
    k0, k1 = np.uint64(int(key[0]) & MASK32), np.uint64(int(key[1]) & MASK32)
    m32 = np.uint64(MASK32)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(WEYL_0)) & m32
            k1 = (k1 + np.uint64(WEYL_1)) & m32
        p0 = np.uint64(MULT_0) * c[0]
        p1 = np.uint64(MULT_1) * c[2]
        hi0, lo0 = (p0 >> np.uint64(32)) & m32, p0 & m32
        hi1, lo1 = (p1 >> np.uint64(32)) & m32, p1 & m32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=1).astype(np.uint32)


def uniform53(words: np.ndarray) -> np.ndarray:
    """FP64 uniform on [0, 1) from two 32-bit words (w0 low, w1 high): top 53 bits * 2^-53."""
    w = words.astype(np.uint64)
    bits = ((w[..., 1] << np.uint64(32)) | w[..., 0]) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53)
