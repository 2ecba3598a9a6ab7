"""GPU: the device Philox-4x32-10 and Gaussian generator against the oracle and cuRAND."""
import numpy as np
import pytest
import torch

from oracle import embedding, philox

pytestmark = pytest.mark.gpu


def test_device_philox_bit_exact_vs_oracle(skel, dev):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64)
    want = philox.philox4x32(ctr, (0x12345678, 0x9ABCDEF0)).astype(np.int64)
    got = skel.debug_philox(torch.from_numpy(ctr.astype(np.int64)).to(dev), 0x12345678, 0x9ABCDEF0)
    assert np.array_equal(got.cpu().numpy(), want)


def test_oracle_philox_matches_curand(skel, dev):
    """cuRAND's Philox4_32_10 (curand_init(seed, subsequence i, offset 0)): its q-th curand4
    output is Philox-4x32-10 of counter (q, 0, i_lo, i_hi) with key (seed_lo, seed_hi).  This
    pins the oracle's 32-bit constants against an independent implementation."""
    seed = 0xDEADBEEF01234567
    nseq, per = 64, 3
    got = skel.debug_curand_philox(seed, nseq, per, device=dev).cpu().numpy()
    ctr = np.array([[q, 0, i & 0xFFFFFFFF, i >> 32] for i in range(nseq) for q in range(per)], dtype=np.uint64)
    want = philox.philox4x32(ctr, philox.seed_key(seed)).astype(np.int64).reshape(nseq, per, 4)
    assert np.array_equal(got, want)


def test_gaussian_fp64_matches_oracle(skel, dev):
    l, m, seed = 37, 1001, 99
    G = skel.debug_gaussian(l, m, seed, fp64=True, device=dev).cpu().numpy()
    want = embedding.gaussian_normals(l, m, seed)
    assert np.max(np.abs(G - want)) < 1e-13


def test_gaussian_fp32_within_ulps(skel, dev):
    """FP32 Box-Muller on the device: within a few FP32 ulps of the FP64 value; after
    rounding to bfloat16 at least 99.9% of the entries are bit-equal to the oracle's."""
    l, m, seed = 64, 4096, 7
    G = skel.debug_gaussian(l, m, seed, fp64=False, device=dev).cpu().numpy().astype(np.float64)
    want = embedding.gaussian_normals(l, m, seed)
    err = np.abs(G - want)
    assert np.all(err <= 8 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0))
    eq = np.mean(embedding.round_bf16(G) == embedding.round_bf16(want))
    assert eq >= 0.999
