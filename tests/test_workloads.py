"""The synthetic inputs follow their recipes: spectra, ranks, shapes and value ranges of the
paper-shaped workloads (small sizes, CPU)."""
import numpy as np
import torch

import workloads


def test_geometric40_spectrum():
    """sigma_j = 10^(-(j-1)/40) plus a 1e-12 Gaussian floor."""
    A = workloads.dense_geometric40(200, 150, seed=1)
    s = np.linalg.svd(A, compute_uv=False)
    want = 10.0 ** (-np.arange(150) / 40.0)
    big = want > 1e-9
    assert np.allclose(s[big], want[big], rtol=1e-6)
    assert A.dtype == np.float64 and A.flags.f_contiguous


def test_harmonic_spectrum_and_floor():
    """sigma_j = 1/j above a noise floor of about 1e-6 (FP32 storage)."""
    m, n = 400, 300
    A = workloads.dense_harmonic(m, n, seed=2, dtype=np.float64)
    s = np.linalg.svd(A, compute_uv=False)
    want = 1.0 / np.arange(1, n + 1)
    assert np.allclose(s[:50], want[:50], rtol=1e-3)
    assert s.min() > 1e-7                       # the floor lifts the tail ...
    A32 = workloads.dense_harmonic(m, n, seed=2)
    assert A32.dtype == np.float32 and A32.flags.f_contiguous


def test_exact_rank_and_haar_factors():
    A = workloads.exact_rank(120, 80, 9, seed=3)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:9], 0.8 ** np.arange(9), rtol=1e-10) and s[9] < 1e-12 * s[0]
    Q = workloads.haar_orthogonal(50, 20, np.random.default_rng(0))
    assert np.allclose(Q.T @ Q, np.eye(20), atol=1e-12)


def test_kernel_blocks_shapes_and_values():
    """Kernel blocks: block sizes inside their ranges, entries exp(-|x-y|^2/h^2) in (0, 1), and
    well-separated clusters make the blocks numerically low rank."""
    blocks = workloads.kernel_blocks(12, seed=4)
    for B in blocks:
        assert 64 <= B.shape[0] <= 1024 and 64 <= B.shape[1] <= 512
        assert B.min() >= 0.0 and B.max() < 1.0 and B.flags.f_contiguous
    s = np.linalg.svd(blocks[0].astype(np.float64), compute_uv=False)
    assert s[60] < 1e-6 * s[0]


def test_torch_builders_match_recipe():
    """The device builders (run here on the CPU) keep the recipe: spectrum of the dense case,
    column-major blocks with 16-byte aligned columns."""
    A = workloads.torch_dense_spectrum(256, 192, workloads.sigma_harmonic(192), 0.0, 5, "cpu", torch.float64)
    s = torch.linalg.svdvals(A).numpy()
    assert np.allclose(s[:40], 1.0 / np.arange(1, 41), rtol=1e-8)
    blocks = workloads.torch_kernel_blocks(6, 7, "cpu")
    for B in blocks:
        assert B.stride(0) == 1 and B.stride(1) % 4 == 0 and B.dtype == torch.float32


def test_snn_is_sparse_nonnegative():
    A = workloads.snn_csc(2000, 500, 50, seed=6)
    assert A.nnz > 0 and A.data.min() >= 0.0
    assert 0.001 < A.nnz / (2000 * 500) < 0.05
