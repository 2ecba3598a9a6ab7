"""Randomized linear embeddings Gamma (l x m) of Sec. 2.3, drawn from Philox-4x32-10.

Gaussian embedding (Sec. 2.3, item 1): i.i.d. entries N(0, 1/l).  Reading: the printed mean
"mu" is taken as 0, as in every cited construction.  The scale 1/sqrt(l) does not change
any pivot (argmax is invariant under positive scaling) and is applied to the sketch.

    counter = (j >> 2, i, TAG_GAUSSIAN, 0), key = seed split in two 32-bit words.
    The four output words (x0, x1, x2, x3) give two Box-Muller pairs, i.e. the four
    standard normals G[i, 4*(j>>2) + q], q = 0..3:
        u_a = (2*(x_a >> 9) + 1) * 2^-24   in [2^-24, 1 - 2^-24] (exact in FP32)
        (G0, G1) = sqrt(-2 ln u_0) * (cos 2 pi u_1, sin 2 pi u_1)
        (G2, G3) = sqrt(-2 ln u_2) * (cos 2 pi u_3, sin 2 pi u_3)
    Gamma = G / sqrt(l).

Sparse sign embedding (Sec. 2.3, item 3): every column s_j of Gamma holds zeta Rademacher
values at uniformly random distinct coordinates.  Readings: coordinates are drawn without
replacement; the printed scale sqrt(m/zeta) is taken as 1/sqrt(zeta), which makes
E[Gamma^T Gamma] = I like the Gaussian embedding (the scale never changes a pivot).

    words w_0, w_1, ... of column j come from counters (j, 0, TAG_SPARSE, c) for
    c = 0, 1, ...; word w_0 holds the signs (bit q set -> the q-th coordinate is -1);
    the coordinates come from Floyd's sampling algorithm (Bentley & Floyd, CACM 1987):
        for q in 0..zeta-1:  J = l - zeta + q;  t = (w_{1+q} * (J + 1)) >> 32
                             take t unless already taken, else take J.
"""

import numpy as np

from .philox import philox4x32, seed_key

TAG_GAUSSIAN = 0
TAG_SPARSE = 1
TAG_SRTT_PERM = 2
TAG_SRTT_SELECT = 3
TAG_SRTT_SIGN = 4


def _unit_open(x):
    """u = (2*(x >> 9) + 1) * 2^-24: 23 random bits, symmetric about 1/2, never 0 or 1."""
    return (2.0 * (x.astype(np.uint64) >> np.uint64(9)).astype(np.float64) + 1.0) * 2.0 ** -24


def gaussian_normals(l, m, seed):
    """Standard normal matrix G (l x m, FP64) with Gamma = G / sqrt(l)."""
    return gaussian_normals_rows(np.arange(l), m, seed)


def gaussian_normals_rows(rows, m, seed):
    """Rows `rows` of G (len(rows) x m): the same counters as gaussian_normals, for sampling
    entries of a large sketch one by one."""
    rows = np.asarray(rows, dtype=np.uint64)
    m4 = (m + 3) // 4
    i_idx, j4_idx = np.meshgrid(rows, np.arange(m4, dtype=np.uint64), indexing="ij")
    ctr = np.zeros((rows.size * m4, 4), dtype=np.uint64)
    ctr[:, 0] = j4_idx.ravel()
    ctr[:, 1] = i_idx.ravel()
    ctr[:, 2] = TAG_GAUSSIAN
    words = philox4x32(ctr, seed_key(seed)).reshape(rows.size, m4, 4)
    G = np.empty((rows.size, m4, 4), dtype=np.float64)
    for a in (0, 2):
        u1 = _unit_open(words[:, :, a])
        u2 = _unit_open(words[:, :, a + 1])
        r = np.sqrt(-2.0 * np.log(u1))
        G[:, :, a] = r * np.cos(2.0 * np.pi * u2)
        G[:, :, a + 1] = r * np.sin(2.0 * np.pi * u2)
    return G.reshape(rows.size, 4 * m4)[:, :m]


def gaussian_embedding(l, m, seed):
    """Gamma (l x m, FP64) with i.i.d. N(0, 1/l) entries (Sec. 2.3, item 1)."""
    return gaussian_normals(l, m, seed) / np.sqrt(l)


def sparse_sign_pattern(l, m, zeta, seed):
    """Coordinates and signs of the sparse sign embedding (Sec. 2.3, item 3).

    returns rows (m x zeta, int64) and signs (m x zeta, +-1.0); column j of Gamma is
    sum_q signs[j, q] / sqrt(zeta) * e_{rows[j, q]}.
    """
    if not (1 <= zeta <= l and zeta <= 31):
        raise ValueError("sparse sign embedding needs 1 <= zeta <= min(l, 31)")
    nw = 1 + zeta
    ncalls = (nw + 3) // 4
    j_idx, c_idx = np.meshgrid(np.arange(m, dtype=np.uint64),
                               np.arange(ncalls, dtype=np.uint64), indexing="ij")
    ctr = np.zeros((m * ncalls, 4), dtype=np.uint64)
    ctr[:, 0] = j_idx.ravel()
    ctr[:, 2] = TAG_SPARSE
    ctr[:, 3] = c_idx.ravel()
    words = philox4x32(ctr, seed_key(seed)).reshape(m, ncalls * 4).astype(np.uint64)
    rows = np.empty((m, zeta), dtype=np.int64)
    for q in range(zeta):                      # Floyd's algorithm, all columns at once
        J = l - zeta + q
        t = ((words[:, 1 + q] * np.uint64(J + 1)) >> np.uint64(32)).astype(np.int64)
        seen = (rows[:, :q] == t[:, None]).any(axis=1) if q else np.zeros(m, dtype=bool)
        rows[:, q] = np.where(seen, J, t)
    sign_bits = words[:, 0]
    signs = np.empty((m, zeta), dtype=np.float64)
    for q in range(zeta):
        signs[:, q] = np.where((sign_bits >> np.uint64(q)) & np.uint64(1), -1.0, 1.0)
    return rows, signs


def sparse_sign_embedding(l, m, zeta, seed):
    """Dense copy of the sparse sign Gamma (l x m, FP64); small sizes only."""
    rows, signs = sparse_sign_pattern(l, m, zeta, seed)
    Gam = np.zeros((l, m), dtype=np.float64)
    cols = np.repeat(np.arange(m), zeta)
    Gam[rows.ravel(), cols] = signs.ravel() / np.sqrt(zeta)
    return Gam


# ---------------------------------------------------------------------------------------
# Subsampled randomized trigonometric transform (Sec. 2.3, item 2):
#     Gamma = sqrt(m/l) Pi_{m->l} T Phi Pi_{m->m}
# with T the unitary discrete Hartley transform of order m (the real trigonometric transform
# the paper names), Phi = diag(phi) Rademacher signs, Pi_{m->m} a random permutation and
# Pi_{m->l} a uniformly random choice of l of the m rows.
#
# Readings.  Conventions: (Pi_{m->m} a)_r = a_{pi(r)} and (Pi_{m->l} d)_i = d_{sel(i)}.
# The random permutation is drawn as a keyed pseudo-random permutation: a balanced 4-round
# Feistel network on 2h bits (Luby & Rackoff, SIAM J. Comput. 1988), 4^h >= m, whose round
# function is Philox word x of the counter (R, round, tag, 0) masked to h bits, mapped onto
# 0..m-1 by cycle walking (Black & Rogaway, CT-RSA 2002: re-apply the network until the value
# falls below m).  The l selected rows are sel(i) = the same construction with another tag,
# i = 0..l-1 (distinct because it is a bijection).  Signs: phi_r = -1 when bit 0 of Philox
# word x of the counter (r, 0, TAG_SRTT_SIGN, 0) is set.  The scale sqrt(m/l) is the
# printed one: with T unitary it makes E[Gamma^T Gamma] = I.
# ---------------------------------------------------------------------------------------
def _feistel_half_bits(m):
    h = 1
    while 4 ** h < m:
        h += 1
    return h


def feistel_permutation(m, seed, tag, x=None):
    """pi(x) for x in 0..m-1 (all of them when x is None): the keyed permutation above."""
    if m < 1 or m > 2 ** 31:
        raise ValueError("1 <= m <= 2^31")
    h = _feistel_half_bits(m)
    mask = np.uint64((1 << h) - 1)
    key = seed_key(seed)
    y = np.arange(m, dtype=np.uint64) if x is None else np.asarray(x, dtype=np.uint64).copy()
    todo = np.ones(y.shape, dtype=bool)
    for _ in range(4 ** h + 1):               # a cycle of the network returns within 4^h steps
        if not todo.any():
            break
        L, R = y[todo] >> np.uint64(h), y[todo] & mask
        for rnd in range(4):
            ctr = np.zeros((R.size, 4), dtype=np.uint64)
            ctr[:, 0] = R
            ctr[:, 1] = rnd
            ctr[:, 2] = tag
            f = philox4x32(ctr, key)[:, 0].astype(np.uint64) & mask
            L, R = R, L ^ f
        y[todo] = (L << np.uint64(h)) | R
        todo = y >= np.uint64(m)
    return y.astype(np.int64)


def srtt_signs(m, seed):
    """phi_r, r = 0..m-1 (+-1.0)."""
    ctr = np.zeros((m, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(m, dtype=np.uint64)
    ctr[:, 2] = TAG_SRTT_SIGN
    w = philox4x32(ctr, seed_key(seed))[:, 0].astype(np.uint64)
    return np.where(w & np.uint64(1), -1.0, 1.0)


def srtt_parts(m, l, seed):
    """(pi, phi, sel) of the SRTT: the permutation, the signs and the l selected rows."""
    if not 1 <= l <= m:
        raise ValueError("the SRTT selects 1 <= l <= m rows")
    return (feistel_permutation(m, seed, TAG_SRTT_PERM), srtt_signs(m, seed),
            feistel_permutation(m, seed, TAG_SRTT_SELECT, np.arange(l)))


def hartley(B):
    """Unitary discrete Hartley transform along axis 0: (T B)_k = m^{-1/2} sum_r
    cas(2 pi k r / m) B_r with cas = cos + sin, taken from the FFT (Re F - Im F, F the
    DFT with kernel exp(-2 pi i k r / m))."""
    B = np.asarray(B, dtype=np.float64)
    F = np.fft.fft(B, axis=0)
    return (F.real - F.imag) / np.sqrt(B.shape[0])


def srtt_apply(A, l, seed):
    """Gamma A for the SRTT, applied in the printed order: permute the rows of A, flip their
    signs, transform, keep the selected rows, scale by sqrt(m/l)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    pi, phi, sel = srtt_parts(m, l, seed)
    B = A[pi] * (phi[:, None] if A.ndim == 2 else phi)
    return np.sqrt(m / l) * hartley(B)[sel]


def srtt_embedding_rows(rows, m, l, seed):
    """Rows `rows` of Gamma (len(rows) x m): row i of T is the transform of e_{sel(i)} (T is
    symmetric), then Gamma(i, pi(r)) = sqrt(m/l) T(sel(i), r) phi_r."""
    pi, phi, sel = srtt_parts(m, l, seed)
    rows = np.asarray(rows, dtype=np.int64)
    E = np.zeros((m, rows.size))
    E[sel[rows], np.arange(rows.size)] = 1.0
    Trows = hartley(E).T                          # len(rows) x m
    G = np.empty_like(Trows)
    G[:, pi] = np.sqrt(m / l) * Trows * phi[None, :]
    return G


def srtt_embedding(l, m, seed):
    """Dense Gamma (l x m) of the SRTT; small sizes only."""
    return srtt_embedding_rows(np.arange(l), m, l, seed)


# ---------------------------------------------------------------------------------------
# Operand rounding, for emulating what a reduced-precision sketch multiplies.
# ---------------------------------------------------------------------------------------

def round_fp32(x):
    """Round to the nearest FP32 value (ties to even), returned as FP64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_e4m3(x):
    """Round to the nearest FP8 e4m3 value (ties to even; 1 sign, 4 exponent bits with bias 7,
    3 mantissa bits; normals from 2^-6, subnormals in steps of 2^-9, largest finite 448),
    saturating at +-448, returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -10)))
    q = 2.0 ** (np.maximum(e, -6.0) - 3.0)              # spacing of the binade (or of subnormals)
    r = np.minimum(np.round(a / q) * q, 448.0)          # numpy rounds halves to even
    return np.copysign(r, x)


def fp8_block_scales(A, block=128):
    """Per-block power-of-two scales of FP8 quantisation: for every `block` consecutive rows of
    each column, s = 2^ceil(log2(amax / 448)) (s = 1 for an all-zero block), the smallest power
    of two that brings the block into e4m3's range.  Returns (ceil(m / block) x n)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    nb = (m + block - 1) // block
    S = np.ones((nb, n))
    for b in range(nb):
        amax = np.abs(A[b * block:(b + 1) * block]).max(axis=0)
        pos = amax > 0
        S[b, pos] = 2.0 ** np.ceil(np.log2(amax[pos] / 448.0))
    return S


def round_fp8_blocks(A, block=128):
    """A rounded to FP8 e4m3 with the per-block power-of-two scales: s * round_e4m3(A / s)."""
    A = np.asarray(A, dtype=np.float64)
    S = np.repeat(fp8_block_scales(A, block), block, axis=0)[:A.shape[0]]
    return S * round_e4m3(A / S)


def round_bf16(x):
    """Round to the nearest bfloat16 value (ties to even) via FP32, returned as FP64.

    bfloat16 keeps the upper 16 bits of an IEEE binary32 word; rounding to nearest even
    adds 0x7FFF plus the lowest kept bit before truncating (finite inputs only).
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    out = (bits << np.uint64(16)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)
