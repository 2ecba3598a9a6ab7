"""Oracle pins for the batched path: the sketch-only column ID (Sec. 4, C^+ A ~ X_1^+ X with the
pseudo-inverse over all l rows of the sketch) and the per-block pipeline with the
tolerance-driven rank."""

import numpy as np
import pytest
from scipy.linalg import solve_triangular

from oracle import decomp, pivoting, rank, sketch, skeleton
import workloads


def _lu_correction_form(X, r):
    """X(:, J)^+ X from the factors of r LUPP steps on all l rows, an independent route:
    X = L R + [0; S] with L = [L_top; L_2] (L_top r x r lower triangular), R(:, J) = R_1 unit
    upper triangular and S(:, J) = 0, so X(:, J) = L R_1 and
        X(:, J)^+ X = R_1^{-1} R + X(0:r, J)^{-1} (I + B^T B)^{-1} B^T S,   B = L_2 L_top^{-1}
    (the truncated solution R_1^{-1} R plus a correction from the rows below the pivots)."""
    piv = pivoting.lupp_columns(X, r)
    Js, L, R = piv["Js"], piv["L"], piv["R"]
    Lt, L2 = L[:r], L[r:]
    S = X[r:] - L2 @ R
    B = solve_triangular(Lt.T, L2.T, lower=False).T          # B L_top = L_2
    G = np.eye(r) + B.T @ B
    corr = np.linalg.solve(X[:r][:, Js], np.linalg.solve(G, B.T @ S))
    return Js, solve_triangular(R[:, Js], R, lower=False, unit_diagonal=True) + corr


def test_sketch_id_interpolates_and_equals_lu_correction_form():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((30, 200))
    r = 12
    Js, Z_lu = _lu_correction_form(X, r)
    Z = decomp.sketch_id(X, Js)
    assert np.allclose(Z[:, Js], np.eye(r), atol=1e-12)
    assert np.allclose(Z, Z_lu, rtol=0, atol=1e-10 * np.abs(Z).max())
    # the normal equations of the sketched least-squares problem hold
    X1 = X[:, Js]
    assert np.linalg.norm(X1.T @ (X - X1 @ Z)) <= 1e-10 * np.linalg.norm(X1) * np.linalg.norm(X)


def test_sketch_id_square_sketch_is_the_printed_inverse():
    """With l = |J_s| (the paper's setting) the pseudo-inverse is the inverse: Z = X_1^{-1} X."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((16, 90))
    Js = pivoting.lupp_columns(X, 16)["Js"]
    Z = decomp.sketch_id(X, Js)
    assert np.allclose(Z, np.linalg.solve(X[:, Js], X), rtol=0, atol=1e-10 * np.abs(Z).max())


def test_sketch_id_uses_the_oversampling_rows():
    """With s < l the rows below the pivots enter Z: the least-squares solution differs from
    the one through the first s rows alone, fits the whole sketch strictly better, and gives a
    smaller ID error on average (sketch-and-solve with oversampling)."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((40, 150))
    Js = pivoting.lupp_columns(X, 25)["Js"]
    Z_ls = decomp.sketch_id(X, Js)
    Z_tr = np.linalg.solve(X[:25][:, Js], X[:25])
    X1 = X[:, Js]
    assert np.linalg.norm(Z_ls - Z_tr) > 1e-3 * np.linalg.norm(Z_tr)
    assert np.linalg.norm(X - X1 @ Z_ls) < np.linalg.norm(X - X1 @ Z_tr)
    r_ls, r_tr = [], []
    for seed in range(12):
        A = workloads.dense_harmonic(300, 200, seed=seed, dtype=np.float64)
        Xs = sketch.gaussian_sketch(A, 40, 100 + seed)
        J = pivoting.lupp_columns(Xs, 25)["Js"]
        C = A[:, J]
        e_opt = np.linalg.norm(A - C @ decomp.column_id(A, J))
        r_ls.append(np.linalg.norm(A - C @ decomp.sketch_id(Xs, J)) / e_opt)
        r_tr.append(np.linalg.norm(A - C @ np.linalg.solve(Xs[:25][:, J], Xs[:25])) / e_opt)
    assert np.mean(r_ls) < np.mean(r_tr)


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
    A = workloads.dense_harmonic(400, 300, seed=9, dtype=np.float64)
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


def test_gaussian_kernel_block_pins():
    """The oracle's kernel block of a point batch: equal to scipy's squared-Euclidean cdist
    route; in 1-D the separable form exp(-x^2/h^2) exp(2xy/h^2) exp(-y^2/h^2); for x = y a
    symmetric positive semidefinite matrix with unit diagonal (the Gaussian kernel is positive
    definite); unchanged when both point sets are translated together."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(21)
    x = rng.random((37, 3)).astype(np.float32)
    y = (rng.random((23, 3)) + np.array([1.5, -0.5, 0.25])).astype(np.float32)
    h = 0.7
    A = skeleton.gaussian_kernel_block(x, y, h)
    ref = np.exp(-cdist(x.astype(np.float64), y.astype(np.float64), "sqeuclidean") / (h * h))
    assert np.allclose(A, ref, rtol=1e-12, atol=0)
    a, b = rng.random(9), rng.random(5) + 0.5
    A1 = skeleton.gaussian_kernel_block(a[:, None], b[:, None], h)
    sep = np.exp(-a ** 2 / h ** 2)[:, None] * np.exp(2 * np.outer(a, b) / h ** 2) * np.exp(-b ** 2 / h ** 2)[None, :]
    assert np.allclose(A1, sep, rtol=1e-12, atol=0)
    K = skeleton.gaussian_kernel_block(x, x, h)
    assert np.array_equal(K, K.T) and np.all(np.diag(K) == 1.0)
    assert np.linalg.eigvalsh(K).min() > -1e-12
    shift = np.array([3.0, -2.0, 0.5])
    At = skeleton.gaussian_kernel_block(x.astype(np.float64) + shift, y.astype(np.float64) + shift, h)
    assert np.allclose(At, A, rtol=1e-9, atol=0)


def test_kernel_points_follow_kernel_blocks():
    """kernel_points draws the same point sets as kernel_blocks (same seed, same order), so the
    oracle's blocks from the FP32 points differ from the FP64-point blocks only by the points'
    rounding (relative 1e-5 at most for exponents down to -130)."""
    pts = workloads.kernel_points(4, seed=8)
    blocks = workloads.kernel_blocks(4, seed=8)
    for (x, y), B in zip(pts, blocks):
        A = skeleton.gaussian_kernel_block(x, y, 0.5)
        assert A.shape == B.shape and x.dtype == np.float32 and x.shape[1] == 3
        nz = B > 1e-30
        assert np.max(np.abs(A[nz] / B[nz] - 1)) < 1e-4
