"""Greedy column pivoting on a row space approximator X (l x n), Sec. 2.5.

Both routines perform the first s greedy steps of the factorization and return the pivot
columns J_s in selection order (0-based; the paper's MATLAB indices are 1-based).

Readings where the paper is silent or garbled:
  * ties: among exactly equal pivot magnitudes the lowest original column index wins;
  * a zero pivot magnitude (rank deficiency; the paper assumes l <= rank) stops the
    factorization with status "rank_deficient" and the steps done so far;
  * the printed Schur-complement update and the R^LU formula of Sec. 2.5.2 carry index
    slips (t versus t+1); the routine below is the standard algorithm they describe
    (Trefethen & Bau, Alg. 21.1, applied to X^T), which gives R^LU(t, j_t) = 1 and
    |R^LU| <= 1 as the section states.
"""

import numpy as np


def _top_two_gap(vals):
    """Relative gap (|best| - |second|) / |best| of a masked magnitude vector."""
    order = np.sort(vals[vals >= 0])[::-1]
    if order.size < 2 or order[0] == 0:
        return 1.0
    return float((order[0] - order[1]) / order[0])


def lupp_columns(X, s):
    """Column-wise LU with partial pivoting on X (Sec. 2.5.2, Eq. (LUPP)).

    Step t (0-based): S is the current Schur complement (rows t.. of X after t steps);
        j_t = argmax over unselected columns j of |S(t, j)|
        L(t:, t)  = S(t:, j_t)
        R(t, :)   = S(t, :) / S(t, j_t)            (R(t, j_t) = 1, |R(t, :)| <= 1)
        S(t+1:, :) -= L(t+1:, t) R(t, :)
    After s steps X(0:s, :) = L(0:s, 0:s) R exactly (in exact arithmetic).

    returns dict(Js (s,), L (l x s), R (s x n), gaps (s,), status, steps)
    """
    S = np.array(X, dtype=np.float64, copy=True)
    l, n = S.shape
    if not (1 <= s <= min(l, n)):
        raise ValueError("need 1 <= s <= min(l, n)")
    avail = np.ones(n, dtype=bool)
    Js = np.full(s, -1, dtype=np.int64)
    L = np.zeros((l, s))
    R = np.zeros((s, n))
    gaps = np.ones(s)
    status = "ok"
    for t in range(s):
        mag = np.where(avail, np.abs(S[t]), -1.0)
        j = int(np.argmax(mag))            # first maximum = lowest index among ties
        if mag[j] == 0.0:
            status = "rank_deficient"
            return dict(Js=Js, L=L, R=R, gaps=gaps, status=status, steps=t)
        gaps[t] = _top_two_gap(mag)
        Js[t] = j
        L[t:, t] = S[t:, j]
        R[t] = S[t] / S[t, j]
        S[t + 1:] -= np.outer(S[t + 1:, j], R[t])
        avail[j] = False
    return dict(Js=Js, L=L, R=R, gaps=gaps, status=status, steps=s)


def lupp_rows(C, s):
    """Row-wise LUPP on C (m x s'): the row pivots of C are the column pivots of C^T
    (Algorithm 2, row pivoting)."""
    return lupp_columns(np.asarray(C).T, s)


def cpqr_columns(X, s):
    """Column pivoted Householder QR on X (Sec. 2.5.1, Eq. (QRCP)), first s steps.

    Step t: j_t = argmax over unselected j of ||S(t:, j)||_2 (norms recomputed exactly);
    a Householder reflector H = I - tau v v^T maps S(t:, j_t) to beta e_1 with
    beta = -sign(S(t, j_t)) ||S(t:, j_t)||, and is applied to every column.
    R(t, :) = S(t, :) after the reflection (R(t, j_t) = beta, R(t, j_{t'}) = 0 for t' < t).

    returns dict(Js, R (s x n), gaps, status, steps)
    """
    S = np.array(X, dtype=np.float64, copy=True)
    l, n = S.shape
    if not (1 <= s <= min(l, n)):
        raise ValueError("need 1 <= s <= min(l, n)")
    avail = np.ones(n, dtype=bool)
    Js = np.full(s, -1, dtype=np.int64)
    R = np.zeros((s, n))
    gaps = np.ones(s)
    for t in range(s):
        norms = np.sqrt(np.sum(S[t:] ** 2, axis=0))
        mag = np.where(avail, norms, -1.0)
        j = int(np.argmax(mag))
        if mag[j] == 0.0:
            return dict(Js=Js, R=R, gaps=gaps, status="rank_deficient", steps=t)
        gaps[t] = _top_two_gap(mag)
        Js[t] = j
        x = S[t:, j].copy()
        alpha = x[0]
        beta = -np.copysign(mag[j], alpha) if alpha != 0 else -mag[j]
        v = x / (alpha - beta)
        v[0] = 1.0
        tau = (beta - alpha) / beta
        S[t:] -= tau * np.outer(v, v @ S[t:])
        S[t + 1:, j] = 0.0                  # exact zeros below the new diagonal entry
        S[t, j] = beta
        R[t] = S[t]
        avail[j] = False
    return dict(Js=Js, R=R, gaps=gaps, status="ok", steps=s)
