"""Pins for the tolerance-driven rank reading (oracle.rank)."""
import numpy as np

from oracle import rank, sketch, pivoting
import workloads


def test_exact_rank_is_found():
    """An exactly rank-r input: the Schur complement vanishes after r steps, so the
    estimate drops to rounding level at t = r and the rule returns rank r."""
    A = workloads.exact_rank(200, 150, 9, seed=1)
    X = sketch.gaussian_sketch(A, 30, seed=2)
    out = rank.lupp_tolerance_rank(X, kmax=20, tol=1e-9)
    assert out["rank"] == 9
    assert np.array_equal(out["Js"], pivoting.lupp_columns(X, 9)["Js"])


def test_estimate_is_unbiased_for_oblique_residual():
    """E ||S_t||_F^2 l/(l-t) = ||A (I - P_t)||_F^2 with P_t = Pi_1 X_1^{-1} X(0:t, :) (proof
    of Theorem 1): the mean ratio over 150 seeds is 1 within sampling error."""
    A = workloads.dense_harmonic(120, 80, seed=3, dtype=np.float64)
    l, t = 20, 8
    ratios = []
    for s in range(150):
        X = sketch.gaussian_sketch(A, l, seed=500 + s)
        piv = pivoting.lupp_columns(X, t)
        Js = piv["Js"]
        n = A.shape[1]
        P = np.zeros((n, n))
        P[Js, :] = np.linalg.solve(X[:t, Js], X[:t])
        resid = np.sum((A - A @ P) ** 2)
        S = X.copy()
        S_t = X[t:] - X[t:, Js] @ np.linalg.solve(X[:t, Js], X[:t])
        est = np.sum(S_t ** 2) * l / (l - t)
        ratios.append(est / resid)
    assert abs(np.mean(ratios) - 1.0) < 0.06


def test_tolerance_monotone():
    A = workloads.dense_harmonic(200, 150, seed=4, dtype=np.float64)
    X = sketch.gaussian_sketch(A, 60, seed=5)
    ranks = [rank.lupp_tolerance_rank(X, kmax=40, tol=tol)["rank"] for tol in (0.5, 0.2, 0.1, 0.05)]
    assert ranks == sorted(ranks) and ranks[0] < ranks[-1]
