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

    returns dict(rank, Js (rank,), estimates (list of the t-th estimate ratio),
                 gaps (relative gap |best| - |second| over |best| of each step taken),
                 mags (|best| of each step taken))
    The steps also stop when no column is left or the best remaining magnitude is 0.
    """
    S = np.array(X, dtype=np.float64, copy=True)
    l, n = S.shape
    if not (1 <= kmax < l):
        raise ValueError("need 1 <= kmax < l")
    normX2 = float(np.sum(S ** 2))
    avail = np.ones(n, dtype=bool)
    Js = []
    ratios = []
    gaps = []
    mags = []
    done = lambda t: dict(rank=t, Js=np.array(Js, dtype=np.int64), estimates=ratios,
                          gaps=np.array(gaps, dtype=np.float64), mags=np.array(mags, dtype=np.float64))
    for t in range(kmax + 1):
        est = float(np.sum(S[t:] ** 2)) * l / (l - t)
        ratios.append(est / normX2 if normX2 > 0 else 0.0)
        if est <= tol * tol * normX2 or t == kmax:
            return done(t)
        mag = np.where(avail, np.abs(S[t]), -1.0)
        j = int(np.argmax(mag))
        if mag[j] <= 0.0:
            return done(t)
        srt = np.sort(mag)
        gaps.append((srt[-1] - max(srt[-2], 0.0)) / srt[-1] if n > 1 else 1.0)
        mags.append(srt[-1])
        Js.append(j)
        r = S[t] / S[t, j]
        S[t + 1:] -= np.outer(S[t + 1:, j], r)
        S[t, :] = 0.0          # row t is eliminated; it no longer belongs to S_{t+1}
        avail[j] = False
    raise AssertionError("unreachable")
