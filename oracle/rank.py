"""Tolerance-driven rank for LUPP on a Gaussian sketch.

The paper fixes the rank k in advance; its algorithms have no tolerance rule.  Reading used
for blocks whose rank is chosen to meet a relative tolerance: after t LUPP steps on
X = Gamma A (l rows), rows t..l-1 of the Schur complement equal Gamma(t:l, :) A (I - P_t),
where P_t is the oblique projector built from the first t rows (proof of Theorem 1) and is
independent of Gamma(t:l, :).  For Gaussian Gamma with N(0, 1/l) entries,
    E ||S_t||_F^2 * l / (l - t) = ||A (I - P_t)||_F^2  >=  ||A - C C^+ A||_F^2,
and ||X||_F^2 estimates ||A||_F^2.  The rank is the smallest t <= k_max with
    ||S_t||_F^2 * l / (l - t) <= tol^2 * ||X||_F^2,
or k_max when no t qualifies.
"""

import numpy as np


def lupp_tolerance_rank(X, kmax, tol):
    """LUPP (same steps as ``pivoting.lupp_columns``) that stops at the tolerance rank.

    returns dict(rank, Js (rank,), estimates (list of the t-th estimate ratio))
    """
    S = np.array(X, dtype=np.float64, copy=True)
    l, n = S.shape
    if not (1 <= kmax < l and kmax <= n):
        raise ValueError("need 1 <= kmax < l and kmax <= n")
    normX2 = float(np.sum(S ** 2))
    avail = np.ones(n, dtype=bool)
    Js = []
    ratios = []
    for t in range(kmax + 1):
        est = float(np.sum(S[t:] ** 2)) * l / (l - t)
        ratios.append(est / normX2 if normX2 > 0 else 0.0)
        if est <= tol * tol * normX2 or t == kmax:
            return dict(rank=t, Js=np.array(Js, dtype=np.int64), estimates=ratios)
        mag = np.where(avail, np.abs(S[t]), -1.0)
        j = int(np.argmax(mag))
        if mag[j] == 0.0:
            return dict(rank=t, Js=np.array(Js, dtype=np.int64), estimates=ratios)
        Js.append(j)
        r = S[t] / S[t, j]
        S[t + 1:] -= np.outer(S[t + 1:, j], r)
        S[t, :] = 0.0          # row t is eliminated; it no longer belongs to S_{t+1}
        avail[j] = False
    raise AssertionError("unreachable")
