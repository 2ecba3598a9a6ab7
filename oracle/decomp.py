"""Interpolative and CUR decompositions from chosen skeletons (Sec. 2.2), and the column ID
formed from the sketch alone (Sec. 4).

Column ID (Eq. (2.1)):   CID(A; J_s) = C C^+ A,  C = A(:, J_s),  so Z = C^+ A.
CUR (Eq. (2.4)):         CUR(A; I_s, J_s) = C (C^+ A R^+) R,  R = A(I_s, :),  U = C^+ A R^+.
Stable CUR (Remark 3):   with C = Q_C R_C and R^T = Q_R R_R (unpivoted QR),
                         CUR = Q_C (Q_C^T A Q_R) Q_R^T,  hence U = R_C^{-1} (Q_C^T A Q_R) R_R^{-T}.

LAPACK Householder QR (numpy.linalg.qr) and triangular solves serve as single steps.
"""

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_triangular


def column_id(A, Js):
    """Z (s x n, FP64) of the column ID A ~ A(:, Js) Z, computed as R_C^{-1} (Q_C^T A)."""
    A = np.asarray(A, dtype=np.float64)
    C = A[:, np.asarray(Js)]
    Q, R = np.linalg.qr(C, mode="reduced")
    return solve_triangular(R, Q.T @ A, lower=False)


def cur(A, Js, Is):
    """U (s x s, FP64) of the CUR A ~ A(:, Js) U A(Is, :) via the stable form (Remark 3).
    A dense, or scipy.sparse (then Q_C^T A Q_R is formed as Q_C^T (A Q_R) with a sparse
    product)."""
    if sp.issparse(A):
        A = A.astype(np.float64)
        C = A[:, np.asarray(Js)].toarray()
        Rm = A.tocsr()[np.asarray(Is), :].toarray()
    else:
        A = np.asarray(A, dtype=np.float64)
        C = A[:, np.asarray(Js)]
        Rm = A[np.asarray(Is), :]
    Qc, Rc = np.linalg.qr(C, mode="reduced")
    Qr, Rr = np.linalg.qr(Rm.T, mode="reduced")
    M = Qc.T @ np.asarray(A @ Qr)
    U = solve_triangular(Rc, M, lower=False)                # R_C^{-1} M
    U = solve_triangular(Rr, U.T, lower=False).T            # (R_R^{-1} U^T)^T = U R_R^{-T}
    return U


def sketch_id(X, Js):
    """Z (s x n) of the column ID estimated from the row sketch without a second pass over A
    (Sec. 4: C^+ A ~ X_1^+ X with X_1 = X(:, J_s)), the pseudo-inverse taken over all l rows of
    the sketch (l >= s = |J_s|):
        Z = X(:, J_s)^+ X = argmin_Z ||X(:, J_s) Z - X||_F = argmin_Z ||Gamma (C Z - A)||_F,
    the sketched least-squares problem for C^+ A.  With l = s it is the paper's X_1^{-1} X.
    A library least-squares solve serves as the step."""
    X = np.asarray(X, dtype=np.float64)
    Js = np.asarray(Js, dtype=np.int64)
    if Js.size == 0:
        return np.zeros((0, X.shape[1]))
    return np.linalg.lstsq(X[:, Js], X, rcond=None)[0]


def cur_sketch(A, Js, Is):
    """U of the CUR estimated without a second pass over A (Sec. 4): with S = A(I_s, J_s),
    A ~ C S^{-1} R, so U = S^{-1} (a library inverse serves as the step)."""
    A = np.asarray(A, dtype=np.float64)
    return np.linalg.inv(A[np.ix_(np.asarray(Is), np.asarray(Js))])
