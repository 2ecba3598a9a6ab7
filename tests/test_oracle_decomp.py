"""Pins for the oracle's column ID, CUR, errors and Theorem 1 (Secs. 2.2, 2.4, 4)."""
import itertools

import numpy as np
import pytest

from oracle import decomp, errors, pivoting, sketch, skeleton
import workloads


def test_id_interpolates_skeleton_columns():
    """Z(:, Js) = I for linearly independent skeleton columns (Eq. (2.1))."""
    A = workloads.dense_geometric40(200, 150, seed=3)
    Js = np.array([5, 17, 3, 100, 42])
    Z = decomp.column_id(A, Js)
    assert np.allclose(Z[:, Js], np.eye(5), atol=1e-10)


def test_id_is_least_squares_optimal():
    """C^T (A - C Z) = 0 (normal equations), and Z equals numpy's lstsq solution."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((80, 60))
    Js = rng.choice(60, 12, replace=False)
    Z = decomp.column_id(A, Js)
    C = A[:, Js]
    assert np.max(np.abs(C.T @ (A - C @ Z))) < 1e-11
    Zl = np.linalg.lstsq(C, A, rcond=None)[0]
    assert np.allclose(Z, Zl, atol=1e-11)


def test_exact_rank_reconstruction():
    """Lemma 1 + Algorithm 2: an exactly rank-r input, l = s = r, is reconstructed exactly
    by both the column ID and the CUR (two-sided ID equals column ID, Sec. 3.3)."""
    A = workloads.exact_rank(300, 200, 15, seed=7)
    out = skeleton.skeletonize(A, k=15, p=0, seed=11)
    assert out["err_id"] < 1e-12
    assert out["err_cur"] < 1e-11
    C = A[:, out["Js"]]
    S = C[out["Is"], :]
    assert np.linalg.cond(S) < 1e8


def test_remark1_sandwich():
    """Remark 1: ||A - CC^+A|| <= ||A - CUR|| <= sqrt(||A - CC^+A||^2 + ||A - AR^+R||^2),
    Frobenius and spectral norms."""
    A = workloads.dense_geometric40(120, 90, seed=4)
    out = skeleton.skeletonize(A, k=20, p=5, seed=2)
    Js, Is, Z, U = out["Js"], out["Is"], out["Z"], out["U"]
    C, Rm = A[:, Js], A[Is, :]
    E_id = A - C @ Z
    E_cur = A - C @ U @ Rm
    E_row = A - A @ np.linalg.pinv(Rm) @ Rm
    for nrm in ("fro", 2):
        a, b, c = (np.linalg.norm(E, nrm) for E in (E_id, E_cur, E_row))
        assert a <= b * (1 + 1e-10)
        assert b <= np.sqrt(a ** 2 + c ** 2) * (1 + 1e-10)


def test_stable_cur_equals_definition():
    """U = R_C^{-1} (Q_C^T A Q_R) R_R^{-T} equals C^+ A R^+ (Eq. (2.4), Remark 3)."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((50, 40))
    Js, Is = rng.choice(40, 7, replace=False), rng.choice(50, 7, replace=False)
    U = decomp.cur(A, Js, Is)
    want = np.linalg.pinv(A[:, Js]) @ A @ np.linalg.pinv(A[Is, :])
    assert np.allclose(U, want, atol=1e-10)


def test_theorem1_bound_and_eta_formula():
    """Theorem 1: ||A - CC^+A||_F <= eta ||A - A Xt^+ Xt||_F with Xt = R^LU(0:s, :), and
    eta = ||I - P_X||_2 for the oblique projector P_X = Pi_1 Xt_1^{-1} Xt (brute force)."""
    for seed in range(5):
        A = workloads.dense_harmonic(150, 120, seed=seed, dtype=np.float64)
        X = sketch.gaussian_sketch(A, 26, seed=100 + seed)
        piv = pivoting.lupp_columns(X, 20)
        Js, R = piv["Js"], piv["R"]
        Z = decomp.column_id(A, Js)
        err = errors.fro(A - A[:, Js] @ Z)
        eta = errors.eta(R, Js)
        assert err <= eta * errors.rangefinder_error(A, R) * (1 + 1e-10)
        n = A.shape[1]
        Pi1 = np.zeros((n, len(Js)))
        Pi1[Js, np.arange(len(Js))] = 1.0
        P = Pi1 @ np.linalg.solve(R[:, Js], R)
        assert eta == pytest.approx(np.linalg.norm(np.eye(n) - P, 2), rel=1e-9)
        # the same bound holds for the row space of the first s rows of X
        assert errors.rangefinder_error(A, R) == pytest.approx(errors.rangefinder_error(A, X[:20]), rel=1e-8)


def test_theorem1_bound_cpqr():
    """Theorem 1 with CPQR pivots, Xt = R^QR(0:s, :)."""
    A = workloads.dense_harmonic(140, 100, seed=9, dtype=np.float64)
    X = sketch.gaussian_sketch(A, 30, seed=1)
    piv = pivoting.cpqr_columns(X, 24)
    Z = decomp.column_id(A, piv["Js"])
    err = errors.fro(A - A[:, piv["Js"]] @ Z)
    assert err <= errors.eta(piv["R"], piv["Js"]) * errors.rangefinder_error(A, piv["R"]) * (1 + 1e-10)


def test_volume_sampling_existence_brute_force():
    """Sec. 2.2.3: some k-subset achieves ||A - CC^+A||_F <= sqrt(1+k) ||A - A_k||_F.
    Brute force over all subsets of a tiny matrix; the algorithm's error is >= that minimum
    and its ID error uses the least-squares optimal Z."""
    rng = np.random.default_rng(5)
    for trial in range(3):
        A = rng.standard_normal((9, 11)) @ np.diag(0.6 ** np.arange(11))
        k = 3
        best = min(errors.fro(A - A[:, list(S)] @ np.linalg.lstsq(A[:, list(S)], A, rcond=None)[0])
                   for S in itertools.combinations(range(11), k))
        assert best <= np.sqrt(1 + k) * errors.best_rank_k_error(A, k) * (1 + 1e-12)
        out = skeleton.skeletonize(A, k=k, p=2, seed=trial, want_cur=False)
        assert out["err_id"] * errors.fro(A) >= best * (1 - 1e-12)


def test_rangefinder_expectation_bound():
    """Eq. (2.7): E||A - A X^+ X||_F^2 <= (l-1)/(l-k-1) ||A - A_k||_F^2 for Gaussian
    sketches (mean over 200 seeds, 10% slack for sampling error)."""
    A = workloads.dense_harmonic(60, 50, seed=1, dtype=np.float64)
    k, l = 6, 12
    vals = [errors.rangefinder_error(A, sketch.gaussian_sketch(A, l, seed=s)) ** 2 for s in range(200)]
    bound = (l - 1) / (l - k - 1) * errors.best_rank_k_error(A, k) ** 2
    assert np.mean(vals) <= 1.1 * bound


def test_sparse_sign_skeleton_runs_and_is_close_to_optimal():
    A = workloads.dense_harmonic(400, 200, seed=2, dtype=np.float64)
    out = skeleton.skeletonize(A, k=20, p=20, seed=4, kind="sparse_sign", zeta=8)
    opt = errors.best_rank_k_error(A, 20) / errors.fro(A)
    assert opt <= out["err_id"] < 3 * opt


def test_streaming_selection_exact_on_exactly_low_rank():
    """Algorithm 3 on an exactly rank-r input with k = r: the CUR from the row sketch's column
    pivots and the column sketch's row pivots reconstructs A (Lemma 1)."""
    A = workloads.exact_rank(250, 180, 12, seed=7)
    out = skeleton.streaming_skeletonize(A, 12, 8, 3, 4)
    C, R = A[:, out["Js"]], A[out["Is"], :]
    assert np.linalg.norm(A - C @ out["U"] @ R) <= 1e-9 * np.linalg.norm(A)


def test_streaming_selection_two_sided_bound():
    """The bound after Algorithm 3 (Sec. 4): ||A - CUR||_F <= eta_X ||A - A Xt^+ Xt||_F +
    eta_Y ||A - Yt^T (Yt^T)^+ A||_F, with Xt, Yt the LU factors of the row and the transposed
    column sketch and eta from each factor."""
    for seed in range(4):
        A = workloads.dense_harmonic(200, 160, seed=seed, dtype=np.float64)
        k = 15
        out = skeleton.streaming_skeletonize(A, k, 10, 10 + seed, 20 + seed)
        err = np.linalg.norm(A - A[:, out["Js"]] @ out["U"] @ A[out["Is"], :])
        ex = errors.eta(out["Rx"], out["Js"]) * errors.rangefinder_error(A, out["Rx"])
        ey = errors.eta(out["Ry"], out["Is"]) * errors.rangefinder_error(A.T, out["Ry"])
        assert err <= (ex + ey) * (1 + 1e-10)


def test_cur_sketch_interpolates_skeletons():
    """C S^{-1} R with S = A(Is, Js) reproduces A's skeleton rows and columns exactly
    (Sec. 4): rows Is give S S^{-1} R = R, columns Js give C S^{-1} S = C.  A transposed or
    permuted S^{-1} fails both (S is neither symmetric nor diagonal here)."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((90, 70))
    Js = rng.choice(70, 9, replace=False)
    Is = rng.choice(90, 9, replace=False)
    U = decomp.cur_sketch(A, Js, Is)
    M = A[:, Js] @ U @ A[Is, :]
    assert np.allclose(M[Is, :], A[Is, :], atol=1e-9)
    assert np.allclose(M[:, Js], A[:, Js], atol=1e-9)


def test_cur_sketch_exact_on_exactly_low_rank():
    """An exactly rank-r input with nonsingular S = A(Is, Js) is reproduced exactly by
    C S^{-1} R (the skeleton decomposition of a rank-r matrix), with the skeletons chosen by
    the sketch path (Algorithm 2)."""
    A = workloads.exact_rank(300, 200, 15, seed=7)
    out = skeleton.skeletonize(A, k=15, p=0, seed=11)
    U = decomp.cur_sketch(A, out["Js"], out["Is"])
    M = A[:, out["Js"]] @ U @ A[out["Is"], :]
    assert np.linalg.norm(A - M) <= 1e-9 * np.linalg.norm(A)


def test_cur_sketch_never_beats_the_optimal_core():
    """U = C^+ A R^+ minimises ||A - C U R||_F over all U (Eq. (2.4)), so the sketch-only
    core S^{-1} is never better; on a decaying spectrum it stays within a modest factor."""
    A = workloads.dense_geometric40(160, 120, seed=5)
    out = skeleton.skeletonize(A, k=20, p=8, seed=2)
    Js, Is = out["Js"], out["Is"]
    C, Rm = A[:, Js], A[Is, :]
    e_opt = np.linalg.norm(A - C @ decomp.cur(A, Js, Is) @ Rm)
    e_sk = np.linalg.norm(A - C @ decomp.cur_sketch(A, Js, Is) @ Rm)
    assert e_opt <= e_sk * (1 + 1e-12)
    assert e_sk <= 1e3 * e_opt


def test_cur_sketch_2x2_closed_form():
    """On a 2 x 2 skeleton the core is the adjugate over the determinant."""
    A = np.array([[1.0, 7.0, 2.0], [3.0, 5.0, 4.0], [6.0, 2.0, 9.0]])
    Js, Is = np.array([2, 0]), np.array([1, 2])
    S = np.array([[4.0, 3.0], [9.0, 6.0]])          # A(Is, Js), written out
    det = 4.0 * 6.0 - 3.0 * 9.0
    want = np.array([[6.0, -3.0], [-9.0, 4.0]]) / det
    assert np.allclose(decomp.cur_sketch(A, Js, Is), want, atol=1e-14)
    assert np.allclose(A[np.ix_(Is, Js)], S)


def test_cur_and_its_error_agree_for_sparse_and_dense_input():
    """The sparse form of the stable CUR and of the direct residual (used for the tall sparse
    configuration) equal the dense forms on the same matrix."""
    import scipy.sparse as sps
    A = workloads.snn_csc(700, 300, 12, seed=6, density=0.1).astype(np.float64)
    Ad = A.toarray()
    k = 10
    X = sketch.sparse_sign_sketch(A, 2 * k, 4, 3)
    Js = pivoting.lupp_columns(X, k)["Js"]
    Is = pivoting.lupp_rows(Ad[:, Js], k)["Js"]
    U_s, U_d = decomp.cur(A, Js, Is), decomp.cur(Ad, Js, Is)
    assert np.allclose(U_s, U_d, rtol=1e-10, atol=1e-12 * np.abs(U_d).max())
    e_s, e_d = errors.rel_cur_error(A, Js, U_d, Is), errors.rel_cur_error(Ad, Js, U_d, Is)
    assert abs(e_s - e_d) <= 1e-12 * max(e_d, 1e-300)
    assert sps.issparse(A)

