"""Algorithm 2 (randomized LUPP skeleton selection) end to end, and its CPQR variant
(Algorithm 1 with CPQR on the sketch), followed by the column ID and the stable CUR.

Readings: the algorithms return |J_s| = l pivots; with a target rank k and oversampling p
(l = k + p, Sec. 2.3), the first s = k greedy pivots form the skeleton.  For LUPP the first
k steps read only rows 0..k-1 of X, so the extra p rows never change LUPP's k pivots; they
do enter CPQR's norms.  Row skeletons I_s come from row-wise LUPP on C = A(:, J_s)
(Algorithm 2, row pivoting).
"""

import numpy as np

from . import sketch, pivoting, decomp, errors, rank


def skeletonize(A, k, p, seed, kind="gaussian", pivot="lupp", zeta=8,
                operand_rounding=None, want_cur=True):
    A = np.asarray(A, dtype=np.float64)
    l = k + p
    if kind == "gaussian":
        X = sketch.gaussian_sketch(A, l, seed, operand_rounding)
    elif kind == "sparse_sign":
        X = sketch.sparse_sign_sketch(A, l, zeta, seed)
    elif kind == "srtt":
        X = sketch.srtt_sketch(A, l, seed)
    else:
        raise ValueError(kind)
    if pivot == "lupp":
        piv = pivoting.lupp_columns(X, k)
    elif pivot == "cpqr":
        piv = pivoting.cpqr_columns(X, k)
    else:
        raise ValueError(pivot)
    Js = piv["Js"]
    out = dict(X=X, Js=Js, pivot=piv, Rfac=piv["R"], gaps=piv["gaps"], status=piv["status"])
    if piv["status"] != "ok":
        return out
    Z = decomp.column_id(A, Js)
    out.update(Z=Z, err_id=errors.rel_id_error(A, Js, Z), eta=errors.eta(piv["R"], Js))
    if want_cur:
        C = A[:, Js]
        rp = pivoting.lupp_rows(C, k)
        Is = rp["Js"]
        U = decomp.cur(A, Js, Is)
        out.update(Is=Is, row_pivot=rp, U=U, err_cur=errors.rel_cur_error(A, Js, U, Is))
    return out


def batch_skeletonize(blocks, kmax, p, tol, seed):
    """Batched blocks (the tolerance-rank reading, see rank.py): per block the Gaussian sketch
    with l = kmax + p rows (one Gamma for every block: columns 0..m_b-1 of the same embedding),
    LUPP stopped at the tolerance rank, and the sketch-only column ID (decomp.sketch_id)."""
    out = []
    for A in blocks:
        A = np.asarray(A, dtype=np.float64)
        X = sketch.gaussian_sketch(A, kmax + p, seed)
        rt = rank.lupp_tolerance_rank(X, kmax, tol)
        out.append(dict(rank=rt["rank"], Js=rt["Js"], Z=decomp.sketch_id(X, rt["Js"]), X=X,
                        gaps=rt["gaps"], mags=rt["mags"], estimates=rt["estimates"]))
    return out


def gaussian_kernel_block(x, y, h):
    """A(i, j) = exp(-||x_i - y_j||^2 / h^2) (the Gaussian kernel between point sets x (m x d)
    and y (n x d)), formed in FP64 from the given coordinates: the implicit matrix of a batch
    given by points (Sec. 1: A is needed only through the entries the method evaluates)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    D2 = np.zeros((x.shape[0], y.shape[0]))
    for c in range(x.shape[1]):
        D2 += (x[:, c][:, None] - y[:, c][None, :]) ** 2
    return np.exp(-D2 / (h * h))


def batch_skeletonize_points(points, h, kmax, p, tol, seed):
    """batch_skeletonize on the Gaussian-kernel blocks of the point sets [(x_b, y_b)]."""
    return batch_skeletonize([gaussian_kernel_block(x, y, h) for x, y in points], kmax, p, tol, seed)


def streaming_skeletonize(A, k, p, seed_gamma, seed_omega):
    """Algorithm 3 (streaming skeleton selection): X = Gamma A and Y = A Omega^T from the same
    pass over A, J_s by column LUPP on X, I_s by row LUPP on Y (column LUPP on Y^T); then the
    CUR with those skeletons (the stable form of Remark 3, which needs A again)."""
    A = np.asarray(A, dtype=np.float64)
    l = k + p
    X = sketch.gaussian_sketch(A, l, seed_gamma)
    Yt = sketch.gaussian_col_sketch(A, l, seed_omega)
    px, py = pivoting.lupp_columns(X, k), pivoting.lupp_columns(Yt, k)
    Js, Is = px["Js"], py["Js"]
    U = decomp.cur(A, Js, Is)
    return dict(X=X, Yt=Yt, Js=Js, Is=Is, Rx=px["R"], Ry=py["R"], gaps_x=px["gaps"], gaps_y=py["gaps"], U=U,
                err_cur=errors.rel_cur_error(A, Js, U, Is))
