"""Error measures of Sec. 2.2.2 and the a-posteriori factor of Theorem 1 (Sec. 4).

Theorem 1: for pivots J_s chosen on a full-row-rank row space approximator X with
X Pi = [X_1, X_2] and X_1 nonsingular,
    ||A - C C^+ A|| <= eta ||A - A X^+ X||,   eta = sqrt(1 + ||X_1^{-1} X_2||_2^2).
The proof's last step shows eta = ||[-X_1^{-1} X_2; I]||_2, which equals
sqrt(1 + ||X_1^{-1} X_2||_2^2) exactly (reading: the printed "<=" for eta is an equality).
With s <= l pivots from LUPP, X~ = R^LU(0:s, :) spans the row space of X(0:s, :), and
X~_1^{-1} X~_2 = R_1^{-1} R_2 (Sec. 4, item 1).
"""

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_triangular


def fro(M):
    return float(np.sqrt(np.sum(np.asarray(M, dtype=np.float64) ** 2)))


def rel_id_error(A, Js, Z):
    """||A - A(:, Js) Z||_F / ||A||_F, residual formed directly (Eq. (2.1))."""
    A = np.asarray(A, dtype=np.float64)
    return fro(A - A[:, np.asarray(Js)] @ Z) / fro(A)


def rel_cur_error(A, Js, U, Is):
    """||A - C U R||_F / ||A||_F with C = A(:, Js), R = A(Is, :) (Eq. (2.4)), the residual
    formed directly.  A dense, or scipy.sparse (the residual then formed 256 columns at a
    time)."""
    if sp.issparse(A):
        A = A.tocsc().astype(np.float64)
        CU = A[:, np.asarray(Js)].toarray() @ U
        Rm = A.tocsr()[np.asarray(Is), :].toarray()
        num = 0.0
        for c0 in range(0, A.shape[1], 256):
            blk = A[:, c0:c0 + 256].toarray() - CU @ Rm[:, c0:c0 + 256]
            num += float(np.sum(blk ** 2))
        return float(np.sqrt(num) / np.sqrt(A.multiply(A).sum()))
    A = np.asarray(A, dtype=np.float64)
    C = A[:, np.asarray(Js)]
    Rm = A[np.asarray(Is), :]
    return fro(A - (C @ U) @ Rm) / fro(A)


def interpolation_T(Rfac, Js):
    """T = R_1^{-1} R_2 (s x (n - s)), R_1 = Rfac(:, Js) (upper triangular in pivot order),
    R_2 = Rfac(:, remaining columns in increasing index order)."""
    Rfac = np.asarray(Rfac, dtype=np.float64)
    Js = np.asarray(Js)
    rest = np.setdiff1d(np.arange(Rfac.shape[1]), Js)
    return solve_triangular(Rfac[:, Js], Rfac[:, rest], lower=False)


def eta(Rfac, Js):
    """Theorem 1's factor sqrt(1 + ||R_1^{-1} R_2||_2^2), spectral norm by SVD."""
    T = interpolation_T(Rfac, Js)
    if T.size == 0:
        return 1.0
    return float(np.sqrt(1.0 + np.linalg.norm(T, 2) ** 2))


def rangefinder_error(A, Xt, ord="fro"):
    """||A - A Xt^+ Xt|| for a full-row-rank Xt (s x n): residual of projecting the rows
    of A onto the row space of Xt (Sec. 2.4)."""
    A = np.asarray(A, dtype=np.float64)
    Q, _ = np.linalg.qr(np.asarray(Xt, dtype=np.float64).T, mode="reduced")
    Res = A - (A @ Q) @ Q.T
    return fro(Res) if ord == "fro" else float(np.linalg.norm(Res, 2))


def best_rank_k_error(A, k, ord="fro"):
    """||A - A_k|| from the singular values (Eckart-Young)."""
    sv = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    tail = sv[k:]
    if ord == "fro":
        return float(np.sqrt(np.sum(tail ** 2)))
    return float(tail[0]) if tail.size else 0.0
