"""Philox4x32-10 counter-based generator (oracle; test infrastructure only).

Written from its published definition (J. Salmon, M. Moraes, R. Dror, D. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter and a
2x32-bit key, ten rounds of two 32x32->64 multiplies with the key bumped by the Weyl
constants between rounds.

The sampling step draws, for sample s and site n, counter (n, s, 0, 0) under key
(seed_lo, seed_hi), and turns the first two output words (x0, x1) into a double
u = ((x0 << 21) | (x1 >> 11)) * 2^-53 in [0, 1).
"""
from __future__ import annotations

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform(seed: int, sample: int, site: int) -> float:
    key = (seed & MASK, (seed >> 32) & MASK)
    x0, x1, _, _ = philox4x32_10((site, sample, 0, 0), key)
    return float(((x0 << 21) | (x1 >> 11))) * 2.0 ** -53
