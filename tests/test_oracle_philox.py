"""Pins for the oracle's Philox generator (Salmon et al., SC'11)."""
import numpy as np
import pytest

from oracle import philox


def test_round_structure_matches_numpy_philox4x64():
    """numpy.random.Philox is an independent Philox-4x64-10; it increments its 256-bit
    counter before each block.  The oracle's 4x64 variant shares the round function and the
    key schedule with the 4x32 variant used everywhere, so a swapped output word, a wrong
    xor partner or a missing key bump would fail here."""
    for key, ctr0 in [((1, 2), 0), ((0xDEADBEEF, 0x12345678ABCDEF), 41), ((0, 0), 7)]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64))
        raw = bg.random_raw(8)
        for blk in range(2):
            want = [int(x) for x in raw[4 * blk: 4 * blk + 4]]
            got = philox.philox4x64_scalar([ctr0 + 1 + blk, 0, 0, 0], key)
            assert got == want


def test_4x32_vectorised_equals_scalar_structure():
    """The vectorised 4x32 routine equals a scalar restatement with Python integers."""
    M, W = philox.PHILOX_M4x32, philox.PHILOX_W32
    rng = np.random.default_rng(0)
    ctrs = rng.integers(0, 2 ** 32, size=(50, 4), dtype=np.uint64)
    key = (0x01234567, 0x89ABCDEF)
    got = philox.philox4x32(ctrs, key)
    for row in range(50):
        c = [int(x) for x in ctrs[row]]
        k = list(key)
        for r in range(10):
            p0, p1 = M[0] * c[0], M[1] * c[2]
            c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & 0xFFFFFFFF, (p0 >> 32) ^ c[3] ^ k[1], p0 & 0xFFFFFFFF]
            k = [(k[0] + W[0]) & 0xFFFFFFFF, (k[1] + W[1]) & 0xFFFFFFFF]
        assert [int(x) for x in got[row]] == c


def test_output_bits_are_uniform():
    """Each output bit is 1 with frequency 1/2 (4e5 words, 6 sigma band)."""
    n = 100_000
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n)
    w = philox.philox4x32(ctr, (7, 9)).ravel().astype(np.uint64)
    bits = np.stack([(w >> np.uint64(b)) & np.uint64(1) for b in range(32)]).mean(axis=1)
    assert np.all(np.abs(bits - 0.5) < 6 * 0.5 / np.sqrt(w.size))


def test_key_and_counter_change_everything():
    a = philox.philox4x32(np.array([[0, 0, 0, 0]]), (0, 0))
    b = philox.philox4x32(np.array([[1, 0, 0, 0]]), (0, 0))
    c = philox.philox4x32(np.array([[0, 0, 0, 0]]), (1, 0))
    assert not np.any(a == b) or np.count_nonzero(a == b) <= 1
    assert not np.any(a == c) or np.count_nonzero(a == c) <= 1
