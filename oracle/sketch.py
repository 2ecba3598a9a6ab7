"""Row sketch X = Gamma A (the sketch step of Algorithms 1 and 2; Table 1).

The sketch is a plain product; the only choices are the embedding and, when emulating a
reduced-precision sketch, the rounding applied to each operand before the exact (FP64)
product.
"""

import numpy as np
import scipy.sparse as sp

from . import embedding


def gaussian_sketch(A, l, seed, operand_rounding=None):
    """X = Gamma A with the Gaussian Gamma (l x m) of ``embedding.gaussian_embedding``.

    operand_rounding: None (exact FP64), "fp32", "bf16" or "fp8" (e4m3; A with one power-of-two
    scale per column, the normals unscaled).  When given, the standard normals
    G and A are each rounded to that format, X = (round(G) @ round(A)) / sqrt(l) in FP64 --
    which is what a kernel multiplying such operands with exact products computes, up to
    its own summation order.
    """
    A = np.asarray(A, dtype=np.float64)
    G = embedding.gaussian_normals(l, A.shape[0], seed)
    if operand_rounding == "fp32":
        G, A = embedding.round_fp32(G), embedding.round_fp32(A)
    elif operand_rounding == "bf16":
        G, A = embedding.round_bf16(G), embedding.round_bf16(A)
    elif operand_rounding == "fp8":
        # e4m3: the normals as they are (x1), A with one power-of-two scale per column (a block
        # of all its rows)
        G, A = embedding.round_e4m3(G), embedding.round_fp8_blocks(A, A.shape[0])
    elif operand_rounding is not None:
        raise ValueError(operand_rounding)
    return (G @ A) / np.sqrt(l)


def gaussian_sketch_rows(A_block, l, seed, row0, operand_rounding=None):
    """Partial sketch of rows row0 .. row0+m_b-1 of a larger A: Gamma(:, row0:row0+m_b) A_block.
    Gamma's columns depend only on their global index, so the partial sketches of a row
    partition sum to the sketch of the whole matrix (the row-partitioned sketch step of Algorithm 2)."""
    A_block = np.asarray(A_block, dtype=np.float64)
    mb = A_block.shape[0]
    G = embedding.gaussian_normals(l, row0 + mb, seed)[:, row0:]
    if operand_rounding == "fp32":
        G, A_block = embedding.round_fp32(G), embedding.round_fp32(A_block)
    elif operand_rounding == "bf16":
        G, A_block = embedding.round_bf16(G), embedding.round_bf16(A_block)
    elif operand_rounding is not None:
        raise ValueError(operand_rounding)
    return (G @ A_block) / np.sqrt(l)


def sparse_sign_sketch_rows(A_block, l, zeta, seed, row0):
    """Partial sparse-sign sketch of rows row0 .. row0+m_b-1 (global column indices of Gamma)."""
    A_block = np.asarray(A_block, dtype=np.float64)
    mb = A_block.shape[0]
    rows, signs = embedding.sparse_sign_pattern(l, row0 + mb, zeta, seed)
    rows, signs = rows[row0:], signs[row0:]
    cols = np.repeat(np.arange(mb), zeta)
    Gam = sp.csr_matrix((signs.ravel() / np.sqrt(zeta), (rows.ravel(), cols)), shape=(l, mb))
    return np.asarray(Gam @ A_block, dtype=np.float64)


def sparse_sign_sketch(A, l, zeta, seed):
    """X = Gamma A with the sparse sign Gamma; A dense (ndarray) or scipy.sparse."""
    m = A.shape[0]
    rows, signs = embedding.sparse_sign_pattern(l, m, zeta, seed)
    cols = np.repeat(np.arange(m), zeta)
    Gam = sp.csr_matrix((signs.ravel() / np.sqrt(zeta), (rows.ravel(), cols)), shape=(l, m))
    X = Gam @ A
    return np.asarray(X.todense() if sp.issparse(X) else X, dtype=np.float64)


def gaussian_sketch_power(A, l, seed, q=1):
    """Row space approximator with q plain power iterations (Sec. 3, Eq. (def_power_iter)):
    X = Omega (A^T A)^q with Omega (l x n) Gaussian N(0, 1/l), the counters of the Gaussian
    embedding over n columns; evaluated as (Omega A^T) A, then (X A^T) A."""
    A = np.asarray(A, dtype=np.float64)
    Om = embedding.gaussian_normals(l, A.shape[1], seed) / np.sqrt(l)
    X = Om
    for _ in range(q):
        X = (X @ A.T) @ A
    return X


def gaussian_col_sketch(A, l, seed):
    """Transposed column sketch of the streaming selection (Algorithm 3): Yt = Omega A^T
    (l x m), i.e. Y = A Omega^T, with Omega (l x n) Gaussian N(0, 1/l) over the counters of the
    Gaussian embedding on n columns."""
    A = np.asarray(A, dtype=np.float64)
    Om = embedding.gaussian_normals(l, A.shape[1], seed) / np.sqrt(l)
    return Om @ A.T


def srtt_sketch(A, l, seed):
    """X = Gamma A for the SRTT embedding (Sec. 2.3, item 2), FP64, by the transform applied
    to A's columns (not through a dense Gamma)."""
    return embedding.srtt_apply(A, l, seed)
