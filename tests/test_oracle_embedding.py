"""Pins for the embeddings of Sec. 2.3 (Gaussian and sparse sign) and operand rounding."""
import numpy as np
import pytest
import torch
from scipy import stats

from oracle import embedding, sketch


def test_gaussian_normals_are_standard_normal():
    """KS test against N(0,1) and the first four moments over 4e5 draws."""
    G = embedding.gaussian_normals(100, 4000, seed=123).ravel()
    assert abs(G.mean()) < 5 / np.sqrt(G.size)
    assert abs(G.var() - 1.0) < 5 * np.sqrt(2.0 / G.size)
    assert abs(stats.skew(G)) < 0.03
    assert abs(stats.kurtosis(G)) < 0.06
    assert stats.kstest(G, "norm").pvalue > 1e-3


def test_gaussian_entries_independent_across_rows_and_columns():
    """Sample correlations between neighbouring entries (within a Box-Muller pair, across
    pairs, across rows) vanish: a reused word or a dropped sin/cos would correlate them."""
    G = embedding.gaussian_normals(64, 4096, seed=5)
    n = G.size / 2
    for a, b in [(G[:, 0::4], G[:, 1::4]), (G[:, 1::4], G[:, 2::4]), (G[:-1], G[1:])]:
        r = np.corrcoef(a.ravel(), b.ravel())[0, 1]
        assert abs(r) < 6 / np.sqrt(min(a.size, n))


def test_gaussian_embedding_is_isometric_in_expectation():
    """E[Gamma^T Gamma] = I_m for i.i.d. N(0, 1/l) entries (Sec. 2.3, item 1): the
    average over seeds of Gamma^T Gamma approaches the identity."""
    l, m, S = 20, 12, 400
    acc = np.zeros((m, m))
    for s in range(S):
        Gam = embedding.gaussian_embedding(l, m, seed=1000 + s)
        acc += Gam.T @ Gam
    acc /= S
    assert np.max(np.abs(acc - np.eye(m))) < 6 * np.sqrt(2.0 / (l * S))


def test_gaussian_is_a_function_of_seed_row_column():
    """Regenerating a sub-block gives the same values (counter-based definition)."""
    G = embedding.gaussian_normals(10, 37, seed=9)
    G2 = embedding.gaussian_normals(10, 40, seed=9)
    assert np.array_equal(G, G2[:, :37])
    G3 = embedding.gaussian_normals(10, 37, seed=10)
    assert not np.any(G == G3)


def test_sparse_sign_columns():
    """Every column has zeta distinct coordinates and values +-1/sqrt(zeta) (Sec. 2.3 item 3)."""
    l, m, zeta = 40, 3000, 8
    rows, signs = embedding.sparse_sign_pattern(l, m, zeta, seed=77)
    assert rows.min() >= 0 and rows.max() < l
    for j in range(m):
        assert len(set(rows[j])) == zeta
    Gam = embedding.sparse_sign_embedding(l, m, zeta, seed=77)
    assert np.allclose(np.count_nonzero(Gam, axis=0), zeta)
    assert np.allclose(np.abs(Gam[Gam != 0]), 1 / np.sqrt(zeta))
    assert np.allclose(np.sum(Gam ** 2, axis=0), 1.0)


def test_sparse_sign_coordinates_uniform_and_signs_balanced():
    """Floyd's algorithm draws a uniform zeta-subset: every coordinate appears with
    frequency zeta/l (chi-square), pairs are uniform too, and signs are fair."""
    l, m, zeta = 16, 40000, 5
    rows, signs = embedding.sparse_sign_pattern(l, m, zeta, seed=3)
    counts = np.bincount(rows.ravel(), minlength=l)
    assert stats.chisquare(counts).pvalue > 1e-4
    pair = np.zeros((l, l))
    for q1 in range(zeta):
        for q2 in range(zeta):
            if q1 != q2:
                np.add.at(pair, (rows[:, q1], rows[:, q2]), 1)
    off = pair[~np.eye(l, dtype=bool)]
    assert stats.chisquare(off).pvalue > 1e-4
    assert abs(signs.mean()) < 6 / np.sqrt(signs.size)


def test_sparse_sign_full_column():
    """zeta = l: every coordinate is taken exactly once."""
    rows, _ = embedding.sparse_sign_pattern(8, 500, 8, seed=1)
    assert np.all(np.sort(rows, axis=1) == np.arange(8)[None, :])


def test_round_bf16_matches_torch():
    """The oracle's bfloat16 rounding equals torch's (an independent routine)."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-20, 20, 100000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(embedding.round_bf16(x), want)


def test_integer_sketch_is_exact_in_every_rounding():
    """Small integers survive FP32 and BF16 rounding, so the sketch of an integer matrix by
    a Rademacher-valued embedding is the exact integer product in every mode."""
    rng = np.random.default_rng(4)
    A = rng.integers(-8, 9, size=(50, 30)).astype(np.float64)
    for mode in (None, "fp32", "bf16"):
        Ar = A if mode is None else (embedding.round_fp32(A) if mode == "fp32" else embedding.round_bf16(A))
        assert np.array_equal(Ar, A)
    X = sketch.sparse_sign_sketch(A, l=16, zeta=16, seed=2) * 4.0     # entries +-1
    assert np.array_equal(X, np.round(X))


def test_sketch_scale_preserves_norms_in_expectation():
    """E||Gamma A||_F^2 = ||A||_F^2 for both embeddings."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((200, 10))
    vals_g, vals_s = [], []
    for s in range(100):
        vals_g.append(np.sum(sketch.gaussian_sketch(A, 30, seed=s) ** 2))
        vals_s.append(np.sum(sketch.sparse_sign_sketch(A, 30, 8, seed=s) ** 2))
    nA = np.sum(A ** 2)
    assert abs(np.mean(vals_g) / nA - 1) < 0.05
    assert abs(np.mean(vals_s) / nA - 1) < 0.05


def test_gaussian_rows_subset_matches_full():
    """The row-sampling generator reproduces the full generator's rows bit for bit."""
    G = embedding.gaussian_normals(40, 301, 9)
    rows = [0, 7, 39, 12]
    assert np.array_equal(embedding.gaussian_normals_rows(rows, 301, 9), G[rows])


def test_power_sketch_through_the_svd():
    """X = Omega (A^T A)^q equals Omega V diag(sigma^(2q)) V^T for A = U diag(sigma) V^T (the
    plain power iteration of Sec. 3 written through the SVD factors), q = 1, 2."""
    rng = np.random.default_rng(3)
    m, n, r = 120, 80, 30
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    sig = 0.9 ** np.arange(r)
    A = (U * sig) @ V.T
    Om = embedding.gaussian_normals(12, n, 4) / np.sqrt(12)
    for q in (1, 2):
        want = (Om @ V) * sig ** (2 * q) @ V.T
        assert np.allclose(sketch.gaussian_sketch_power(A, 12, 4, q), want, rtol=0, atol=1e-12)


def test_power_sketch_improves_the_rangefinder_on_a_flat_spectrum():
    """One plain power iteration lowers the rangefinder error ||A - A X^+ X|| on a slowly
    decaying spectrum (the paper's observation for Rand-LUPP-1piter), on average over seeds."""
    from oracle import errors
    import workloads
    A = workloads.dense_spectrum(300, 200, 1.0 / np.sqrt(np.arange(1, 201)), 0.0, seed=9)
    plain = np.mean([errors.rangefinder_error(A, sketch.gaussian_sketch(A, 20, s)) for s in range(8)])
    power = np.mean([errors.rangefinder_error(A, sketch.gaussian_sketch_power(A, 20, s, 1)) for s in range(8)])
    assert power < 0.9 * plain


def test_round_e4m3_matches_torch():
    """e4m3 rounding (ties to even, subnormals) against torch's float8_e4m3fn conversion on
    in-range values, including exact halfway cases; saturation at 448."""
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-3, 2.4, 20000),
                        [0.0, 1.0625, 1.1875, 2.0 ** -7, 3 * 2.0 ** -10, 448.0, -448.0, 15.5, 17.0]])
    x = x[np.abs(x) <= 448.0]
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(embedding.round_e4m3(x), want)
    assert embedding.round_e4m3(np.array([500.0, -1e6]))[0] == 448.0
    assert embedding.round_e4m3(np.array([-1e6]))[0] == -448.0


def test_fp8_block_scales_are_minimal_powers_of_two():
    """s = 2^ceil(log2(amax/448)): |A/s| <= 448 on every block, and s/2 would overflow."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((300, 20)) * 10.0 ** rng.uniform(-5, 5, (1, 20))
    A[:, 3] = 0.0
    S = embedding.fp8_block_scales(A)
    assert S.shape == (3, 20) and np.all(S[:, 3] == 1.0)
    for b in range(3):
        amax = np.abs(A[b * 128:(b + 1) * 128]).max(axis=0)
        nz = amax > 0
        assert np.all(np.log2(S[b]) == np.round(np.log2(S[b])))
        assert np.all(amax[nz] / S[b, nz] <= 448.0)
        assert np.all(amax[nz] / (S[b, nz] / 2) > 448.0)
    R = embedding.round_fp8_blocks(A)
    assert np.all(np.abs(R - A) <= 2.0 ** -4 * np.abs(A) + 2.0 ** -9 * np.repeat(S, 128, axis=0)[:300])


@pytest.mark.parametrize("m", [1, 2, 3, 5, 16, 17, 1000, 4096, 4097])
def test_feistel_permutation_is_a_bijection(m):
    """The keyed permutation (Feistel network + cycle walking) hits every index once, for
    domains that are and are not powers of 4."""
    for tag in (embedding.TAG_SRTT_PERM, embedding.TAG_SRTT_SELECT):
        pi = embedding.feistel_permutation(m, 7, tag)
        assert np.array_equal(np.sort(pi), np.arange(m))
    sub = embedding.feistel_permutation(m, 7, embedding.TAG_SRTT_PERM, np.arange(m)[::-1])
    assert np.array_equal(sub, embedding.feistel_permutation(m, 7, embedding.TAG_SRTT_PERM)[::-1])


def test_feistel_permutation_depends_on_seed_and_tag():
    a = embedding.feistel_permutation(4096, 1, embedding.TAG_SRTT_PERM)
    b = embedding.feistel_permutation(4096, 2, embedding.TAG_SRTT_PERM)
    c = embedding.feistel_permutation(4096, 1, embedding.TAG_SRTT_SELECT)
    assert np.mean(a == b) < 0.01 and np.mean(a == c) < 0.01
    # a random permutation has ~1 fixed point and its positions are uncorrelated with values
    assert np.sum(a == np.arange(4096)) < 10
    assert abs(np.corrcoef(a, np.arange(4096))[0, 1]) < 0.1


def test_hartley_transform_closed_forms():
    """The unitary DHT is its own inverse, and on e_1 at k = m/4 it gives cas(pi/2)/sqrt(m) =
    +1/sqrt(m) (a flipped sine, cas(-theta) = cos - sin, would give -1/sqrt(m)); the
    transform of a constant vector is sqrt(m) e_0 times that constant."""
    rng = np.random.default_rng(3)
    for m in (1, 2, 7, 64, 1000):
        x = rng.standard_normal((m, 3))
        assert np.allclose(embedding.hartley(embedding.hartley(x)), x, atol=1e-12)
        assert np.isclose(np.linalg.norm(embedding.hartley(x)), np.linalg.norm(x))
    m = 64
    e1 = np.zeros(m)
    e1[1] = 1.0
    t = embedding.hartley(e1)
    assert np.isclose(t[m // 4], 1.0 / np.sqrt(m)) and np.isclose(t[3 * m // 4], -1.0 / np.sqrt(m))
    assert np.isclose(t[0], 1.0 / np.sqrt(m)) and np.isclose(t[m // 8], np.sqrt(2.0) / np.sqrt(m))
    c = embedding.hartley(np.full(m, 2.0))
    assert np.isclose(c[0], 2.0 * np.sqrt(m)) and np.allclose(c[1:], 0.0, atol=1e-12)


def test_srtt_full_selection_is_orthogonal():
    """With l = m the SRTT is sqrt(1) T Phi Pi (all rows kept, permuted): an orthogonal
    matrix, so Gamma^T Gamma = I to rounding."""
    for m in (5, 64, 300):
        G = embedding.srtt_embedding(m, m, 11)
        assert np.allclose(G.T @ G, np.eye(m), atol=1e-12)


def test_srtt_dense_rows_agree_with_the_transform():
    """The dense Gamma (rows of T scattered through the permutation) applied to A equals the
    transform applied to A's columns in the printed order; any row subset agrees too."""
    rng = np.random.default_rng(5)
    m, l = 300, 40
    A = rng.standard_normal((m, 25))
    G = embedding.srtt_embedding(l, m, 9)
    assert np.allclose(G @ A, sketch.srtt_sketch(A, l, 9), atol=1e-12)
    rows = np.array([3, 0, 39, 17])
    assert np.allclose(embedding.srtt_embedding_rows(rows, m, l, 9), G[rows], atol=1e-14)
    # entries have modulus <= sqrt(2/l) (|cas| <= sqrt 2), and row norms are sqrt(m/l)
    assert np.abs(G).max() <= np.sqrt(2.0 / l) * (1 + 1e-12)
    assert np.allclose(np.linalg.norm(G, axis=1), np.sqrt(m / l))


def test_srtt_is_isometric_in_expectation():
    """E ||Gamma x||^2 = ||x||^2 over the random choices (T unitary, l of m rows, scale m/l)."""
    rng = np.random.default_rng(6)
    m, l = 256, 32
    x = rng.standard_normal(m)
    vals = [np.sum(sketch.srtt_sketch(x[:, None], l, s) ** 2) for s in range(400)]
    assert abs(np.mean(vals) / np.sum(x ** 2) - 1.0) < 0.05
    phi = embedding.srtt_signs(4096, 3)
    assert set(np.unique(phi)) == {-1.0, 1.0} and abs(np.mean(phi)) < 0.05


def test_srtt_skeleton_exact_on_exactly_low_rank():
    """Algorithm 2 with the SRTT sketch reconstructs an exactly rank-r input (l >= r)."""
    import workloads
    from oracle import skeleton
    A = workloads.exact_rank(300, 200, 15, seed=7)
    out = skeleton.skeletonize(A, k=15, p=5, seed=11, kind="srtt")
    assert out["err_id"] < 1e-12


def test_srtt_entries_closed_form():
    """Multiplying out sqrt(m/l) Pi_{m->l} T Phi Pi_{m->m} gives, entry by entry,
    Gamma(i, q) = phi_r cas(2 pi sel(i) r / m) / sqrt(l) with r = pi^{-1}(q); the oracle's
    FFT route agrees with it (m not a power of two included)."""
    for m, l in ((300, 40), (256, 256), (97, 13)):
        pi, phi, sel = embedding.srtt_parts(m, l, 21)
        rinv = np.empty(m, dtype=np.int64)
        rinv[pi] = np.arange(m)
        ang = 2.0 * np.pi * ((sel[:, None] * rinv[None, :]) % m) / m
        want = phi[rinv][None, :] * (np.cos(ang) + np.sin(ang)) / np.sqrt(l)
        assert np.allclose(embedding.srtt_embedding(l, m, 21), want, atol=1e-13)


def test_column_sketch_definition_and_range():
    """Y = A Omega^T (Algorithm 3's column sketch) is the row sketch of A^T with the same
    Omega, and on an exactly rank-r input with l >= r its columns span the range of A."""
    import workloads
    rng = np.random.default_rng(9)
    A = rng.standard_normal((60, 45))
    Yt = sketch.gaussian_col_sketch(A, 12, 5)
    assert Yt.shape == (12, 60)
    assert np.allclose(Yt, sketch.gaussian_sketch(A.T, 12, 5), atol=1e-13)
    B = workloads.exact_rank(120, 90, 7, seed=2)
    Y = sketch.gaussian_col_sketch(B, 10, 3).T                     # 120 x 10
    Q, _ = np.linalg.qr(Y)
    assert np.linalg.norm(B - Q @ (Q.T @ B)) <= 1e-10 * np.linalg.norm(B)
