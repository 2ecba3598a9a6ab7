"""Pins for the oracle's LUPP and CPQR (Sec. 2.5) and the Lemma 2 worked case."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import pivoting, errors
import workloads


def _tie_free(l, n, seed):
    return np.random.default_rng(seed).standard_normal((l, n))


@pytest.mark.parametrize("l,n,s", [(12, 40, 12), (30, 200, 20), (64, 64, 64)])
def test_lupp_equals_lapack_getrf_on_transpose(l, n, s):
    """Column-wise LUPP on X is row-pivoted LU of X^T: LAPACK getrf's first s pivot rows
    (sequential swaps replayed) equal J_s on tie-free input."""
    X = _tie_free(l, n, seed=l + n)
    out = pivoting.lupp_columns(X, s)
    _, piv = sla.lu_factor(X.T)
    perm = np.arange(n)
    for i, p in enumerate(piv):
        perm[i], perm[p] = perm[p], perm[i]
    assert np.array_equal(out["Js"], perm[:s])


def test_lupp_factor_properties():
    """R(t, j_t) = 1, |R| <= 1, R strictly lower part zero in pivot order, and
    X(0:s, :) = L(0:s, 0:s) R (Sec. 2.5.2)."""
    X = _tie_free(25, 300, seed=1)
    s = 20
    out = pivoting.lupp_columns(X, s)
    Js, L, R = out["Js"], out["L"], out["R"]
    assert np.allclose(R[np.arange(s), Js], 1.0)
    assert np.max(np.abs(R)) <= 1.0 + 1e-15
    R1 = R[:, Js]
    assert np.array_equal(np.tril(R1, -1), np.zeros((s, s)))
    assert np.allclose(L[:s, :s] @ R, X[:s], atol=1e-12 * np.abs(X).max())
    assert np.array_equal(np.triu(L[:s, :s], 1), np.zeros((s, s)))


def test_lupp_prefix_independent_of_extra_rows():
    """The first k LUPP steps read only rows 0..k-1: pivots on X(0:k, :) and on X agree."""
    X = _tie_free(40, 500, seed=2)
    k = 30
    a = pivoting.lupp_columns(X, k)["Js"]
    b = pivoting.lupp_columns(X[:k], k)["Js"]
    assert np.array_equal(a, b)


def test_lupp_tie_break_lowest_index(golden_dir):
    """Lemma 2's Kahan-type X = [R_1, R_2] has all |entries| = 1 in row 0 and ties at every
    step; lowest-index tie-breaking reproduces R_1, R_2 exactly and the growth
    max |(R_1^{-1} R_2)_{ij}| = 2^(l-i) printed in Lemma 2 (golden fixture)."""
    want = np.loadtxt(f"{golden_dir}/lemma2_kahan_l6.txt")
    l, n = 6, 9
    X = workloads.kahan_type(l, n)
    out = pivoting.lupp_columns(X, l)
    assert np.array_equal(out["Js"], np.arange(l))
    assert np.array_equal(out["R"], X)
    T = errors.interpolation_T(out["R"], out["Js"])
    assert np.array_equal(T, want)
    assert errors.eta(out["R"], out["Js"]) == pytest.approx(np.sqrt(1 + np.linalg.norm(want, 2) ** 2))


def test_lupp_rank_deficient_stops():
    """Rank-2 X: the third pivot magnitude is exactly zero -> status rank_deficient."""
    X = np.zeros((4, 6))
    X[0, 1] = 2.0
    X[1, 3] = -1.0
    out = pivoting.lupp_columns(X, 4)
    assert out["status"] == "rank_deficient" and out["steps"] == 2
    assert list(out["Js"][:2]) == [1, 3]


@pytest.mark.parametrize("l,n,s", [(10, 50, 10), (24, 150, 16)])
def test_cpqr_equals_lapack_geqp3(l, n, s):
    """CPQR's J_s equals LAPACK geqp3's first s pivots on tie-free input, and the diagonal
    |R(t, j_t)| equals |R_lapack(t, t)| (non-increasing)."""
    X = _tie_free(l, n, seed=3 * l + n)
    out = pivoting.cpqr_columns(X, s)
    Q, Rl, P = sla.qr(X, pivoting=True, mode="economic")
    assert np.array_equal(out["Js"], P[:s])
    diag = np.abs(out["R"][np.arange(s), out["Js"]])
    assert np.allclose(diag, np.abs(np.diag(Rl))[:s], rtol=1e-10)
    assert np.all(np.diff(diag) <= 1e-12)


def test_cpqr_factor_reconstructs():
    """X(:, Js) = Q R(:, Js) with R upper triangular in pivot order: R^T R on the pivot
    columns equals X(:, Js)^T X(:, Js) (Q orthonormal), for s = l."""
    X = _tie_free(8, 30, seed=4)
    out = pivoting.cpqr_columns(X, 8)
    R1 = out["R"][:, out["Js"]]
    assert np.allclose(np.tril(R1, -1), 0)
    XJ = X[:, out["Js"]]
    assert np.allclose(R1.T @ R1, XJ.T @ XJ, atol=1e-12)
    assert np.allclose(out["R"].T @ out["R"], X.T @ X, atol=1e-11)


def test_lupp_and_cpqr_on_row_pivots():
    """Row-wise LUPP on C equals column-wise LUPP on C^T (Algorithm 2, row pivoting)."""
    C = _tie_free(60, 9, seed=5)
    assert np.array_equal(pivoting.lupp_rows(C, 9)["Js"], pivoting.lupp_columns(C.T, 9)["Js"])
