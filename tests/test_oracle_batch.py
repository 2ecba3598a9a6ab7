"""Oracle pins for the batched path: the sketch-only column ID (Sec. 4, C^+ A ~ X_1^+ X on the
first r rows of the sketch) and the per-block pipeline with the tolerance-driven rank."""

import numpy as np
import pytest
from scipy.linalg import solve_triangular

from oracle import decomp, pivoting, rank, sketch, skeleton
import workloads


def test_sketch_id_interpolates_and_equals_lu_form():
    """Z(:, Js) = I, and Z equals R_1^{-1} R formed from the LUPP factor (an independent route:
    X(0:r, :) = L R with R(:, Js) unit upper triangular)."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((30, 200))
    r = 12
    piv = pivoting.lupp_columns(X, r)
    Js = piv["Js"]
    Z = decomp.sketch_id(X, Js)
    assert np.allclose(Z[:, Js], np.eye(r), atol=1e-12)
    R = piv["R"]
    Z_lu = solve_triangular(R[:, Js], R, lower=False, unit_diagonal=True)
    assert np.allclose(Z, Z_lu, rtol=0, atol=1e-10 * np.abs(Z).max())


def test_sketch_id_exact_on_exactly_low_rank_input():
    """rank(A) = r: the tolerance rule stops at r and A = A(:, J) Z exactly (the row space of
    X(0:r, :) is A's)."""
    A = workloads.exact_rank(300, 180, 9, seed=5)
    out = skeleton.batch_skeletonize([A], kmax=20, p=10, tol=1e-8, seed=3)[0]
    assert out["rank"] == 9
    res = np.linalg.norm(A - A[:, out["Js"]] @ out["Z"]) / np.linalg.norm(A)
    assert res < 1e-10


def test_sketch_id_not_better_than_least_squares():
    """C^+ A minimises ||A - C Z||_F: the sketch-only Z can only do worse (or equal)."""
    rng = np.random.default_rng(2)
    A = workloads.dense_config2(400, 300, seed=9, dtype=np.float64)
    l, k = 40, 25
    X = sketch.gaussian_sketch(A, l, 4)
    Js = pivoting.lupp_columns(X, k)["Js"]
    C = A[:, Js]
    e_sk = np.linalg.norm(A - C @ decomp.sketch_id(X, Js))
    e_ls = np.linalg.norm(A - C @ decomp.column_id(A, Js))
    assert e_sk >= e_ls * (1 - 1e-12)


def test_tolerance_rank_stops_without_columns():
    """More steps than columns: the steps end when no column is left."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 7))
    out = rank.lupp_tolerance_rank(X, kmax=20, tol=0.0)
    assert out["rank"] == 7 and sorted(out["Js"]) == list(range(7))
    assert len(out["gaps"]) == 7


def test_kernel_blocks_reach_tolerance():
    """Config-4 style blocks (Gaussian kernel between separated clusters) are numerically low
    rank: the estimated relative error at the chosen rank meets the tolerance and the
    sketch-only ID's actual error is of that order."""
    blocks = workloads.kernel_blocks(6, seed=11, mrange=(64, 300), nrange=(64, 300))
    outs = skeleton.batch_skeletonize(blocks, kmax=64, p=16, tol=1e-6, seed=2)
    for A, o in zip(blocks, outs):
        A = A.astype(np.float64)
        assert o["rank"] < 64
        assert o["estimates"][o["rank"]] <= 1e-12
        e = np.linalg.norm(A - A[:, o["Js"]] @ o["Z"]) / np.linalg.norm(A)
        assert e < 1e-4
