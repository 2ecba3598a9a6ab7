"""Philox counter-based generator, written from its published definition.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11.  Philox-4xW-R maps a counter of four W-bit words and a key of
two W-bit words through R rounds.  One round:

    (hi0, lo0) = mulhilo(M0, c0)        (hi1, lo1) = mulhilo(M1, c2)
    c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)

and between rounds the key is bumped by the Weyl constants (k0 += W0, k1 += W1).

The paper draws its embeddings from unspecified generators (Sec. 2.3); this implementation
fixes Philox-4x32-10 as the counter-based source of every random number the method draws, so
that the GPU can regenerate any entry of Gamma from (seed, row, column) without storing it.
"""

import numpy as np

# Published round multipliers and Weyl key increments.
PHILOX_M4x32 = (0xD2511F53, 0xCD9E8D57)
PHILOX_W32 = (0x9E3779B9, 0xBB67AE85)
PHILOX_M4x64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
PHILOX_W64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox4x32(counters, key, rounds=10):
    """Philox-4x32-R on an array of counters.

    counters : uint32 array of shape (N, 4)
    key      : (k0, k1) python ints (32-bit each)
    returns  : uint32 array of shape (N, 4)
    """
    c = np.asarray(counters, dtype=np.uint64) & 0xFFFFFFFF
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0 = np.uint64(key[0] & 0xFFFFFFFF)
    k1 = np.uint64(key[1] & 0xFFFFFFFF)
    m0 = np.uint64(PHILOX_M4x32[0])
    m1 = np.uint64(PHILOX_M4x32[1])
    lo_mask = np.uint64(0xFFFFFFFF)
    for r in range(rounds):
        p0 = m0 * c0            # 32 x 32 -> 64 bit product, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & lo_mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & lo_mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r + 1 < rounds:
            k0 = (k0 + np.uint64(PHILOX_W32[0])) & lo_mask
            k1 = (k1 + np.uint64(PHILOX_W32[1])) & lo_mask
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def philox4x64_scalar(counter, key, rounds=10):
    """Philox-4x64-R on one counter, with Python integers (slow; used only to pin the round
    structure shared with the 4x32 variant against an independent implementation)."""
    mask = (1 << 64) - 1
    c = [int(x) & mask for x in counter]
    k = [int(x) & mask for x in key]
    for r in range(rounds):
        p0 = PHILOX_M4x64[0] * c[0]
        p1 = PHILOX_M4x64[1] * c[2]
        hi0, lo0 = p0 >> 64, p0 & mask
        hi1, lo1 = p1 >> 64, p1 & mask
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        if r + 1 < rounds:
            k = [(k[0] + PHILOX_W64[0]) & mask, (k[1] + PHILOX_W64[1]) & mask]
    return c


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit key words (low word first)."""
    seed = int(seed) & ((1 << 64) - 1)
    return (seed & 0xFFFFFFFF, seed >> 32)
