"""Row-partitioned sketch across ranks (one process per GPU).

The sketch X = Gamma A (Algorithm 2, sketch step) is a sum over the rows of A: with A's rows split
into blocks, X = sum_r Gamma(:, rows_r) A(rows_r, :).  Gamma is counter-based (its column j
depends only on the seed and j), so each rank generates exactly the columns of Gamma that
meet its rows and the partial sketches need one exchange: a sum all-reduce of the l x n
result.  Pivoting and everything after it then run on the reduced X on every rank (or on one).

Host logic only; the partial sketch itself is `paper_2104_05877_gb300.sketch(..., row0=...)`.
"""

import torch
import torch.distributed as tdist


def row_partition(m, world, align=32):
    """Split rows 0 .. m-1 into `world` contiguous blocks (row0, rows) whose starts are
    multiples of `align` (the Gaussian generator consumes Gamma columns in groups of 4, the
    tensor-core kernel in K-steps of 32).  Block sizes differ by at most `align`; trailing
    blocks may be empty when m is small."""
    if world < 1 or align < 4 or align % 4:
        raise ValueError("world >= 1 and align a positive multiple of 4")
    units = (m + align - 1) // align
    base, extra = divmod(units, world)
    out, r0 = [], 0
    for r in range(world):
        u = base + (1 if r < extra else 0)
        rows = max(0, min(m, r0 + u * align) - r0)
        out.append((r0, rows))
        r0 += rows
    return out


def allreduce_partial(X, group=None):
    """Sum the ranks' partial sketches in place (the single exchange step)."""
    if tdist.is_available() and tdist.is_initialized():
        tdist.all_reduce(X, op=tdist.ReduceOp.SUM, group=group)
    return X


def sketch_allreduce(A_local, row0, l, kind="gaussian", prec="tf32", seed=0, zeta=8, group=None, status=None):
    """This rank's partial sketch of rows row0 .. row0+m_local-1, summed over the group:
    every rank returns the sketch of the whole A."""
    from . import new_status, sketch

    if A_local.shape[0] == 0:            # an empty block contributes zeros
        X = torch.zeros(l, A_local.shape[1], dtype=torch.float64 if prec == "f64" else torch.float32,
                        device=A_local.device)
        return allreduce_partial(X, group), (status if status is not None else new_status(A_local.device))
    X, st = sketch(A_local, l, kind=kind, prec=prec, seed=seed, zeta=zeta, status=status, row0=row0)
    return allreduce_partial(X, group), st      # NCCL: ordered on the current stream
