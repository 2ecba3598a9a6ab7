"""GPU: the sketch X = Gamma A against the oracle (Algorithm 2, sketch step)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import embedding, pivoting, sketch
import workloads

pytestmark = pytest.mark.gpu


def _bound(l, m, seed, A, u):
    """Elementwise bound m*u*(|G| |A|)/sqrt(l) on the summation-order difference."""
    G = embedding.gaussian_normals(l, m, seed)
    return (m * u + 1e-15) * (np.abs(G) @ np.abs(A)) / np.sqrt(l) + 1e-300


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1000, 777, 61), (129, 1, 5), (64, 300, 1)])
def test_sketch_fp64(skel, dev, m, n, l):
    A = workloads.dense_geometric40(m, n, seed=m + n) if m >= n else np.random.default_rng(1).standard_normal((m, n))
    A = np.asfortranarray(A)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="f64", seed=42)
    skel.check_status(st)
    want = sketch.gaussian_sketch(A, l, 42)
    assert np.all(np.abs(X.cpu().numpy() - want) <= _bound(l, m, 42, A, 2.0 ** -52))


@pytest.mark.parametrize("m,n,l", [(512, 300, 40), (1000, 130, 80)])
def test_sketch_fp32(skel, dev, m, n, l):
    A = workloads.dense_harmonic(m, n, seed=3)                 # FP32 storage
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="f32", seed=5)
    skel.check_status(st)
    want = sketch.gaussian_sketch(A.astype(np.float64), l, 5, operand_rounding="fp32")
    bound = _bound(l, m, 5, A.astype(np.float64), 2.0 ** -23) + 8 * 2.0 ** -24 * _bound(l, m, 5, A, 1.0) / m
    assert np.all(np.abs(X.cpu().numpy() - want) <= bound)


def test_sketch_empty_and_zero_m(skel, dev):
    A = torch.zeros(0, 5, dtype=torch.float64, device=dev)
    X, st = skel.sketch(A, 3, prec="f64")
    skel.check_status(st)
    assert torch.all(X == 0)


def test_sketch_nonfinite_reported(skel, dev):
    A = np.random.default_rng(0).standard_normal((50, 40))
    A[7, 3] = np.nan
    _, st = skel.sketch(torch.from_numpy(np.asfortranarray(A)).to(dev), 8, prec="f64")
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 3


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sparse_sign_dense_input(skel, dev, dtype):
    m, n, l, zeta = 700, 150, 48, 8
    A = np.asfortranarray(np.random.default_rng(2).standard_normal((m, n)).astype(dtype))
    prec = "f64" if dtype == np.float64 else "f32"
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, kind="sparse_sign", prec=prec, seed=11, zeta=zeta)
    skel.check_status(st)
    want = sketch.sparse_sign_sketch(A.astype(np.float64), l, zeta, 11)
    u = 2.0 ** -52 if dtype == np.float64 else 2.0 ** -23
    Gam = embedding.sparse_sign_embedding(l, m, zeta, 11)
    bound = m * u * (np.abs(Gam) @ np.abs(A.astype(np.float64))) + 1e-300
    assert np.all(np.abs(X.cpu().numpy() - want) <= bound)


def test_sparse_sign_pattern_is_exact(skel, dev):
    """Integer A with zeta = l: X = sum of signed entries, exact in FP64; checks every
    (row, sign) of the device pattern against the oracle's."""
    m, n, l = 300, 64, 8
    A = np.asfortranarray(np.random.default_rng(5).integers(-4, 5, size=(m, n)).astype(np.float64))
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, kind="sparse_sign", prec="f64", seed=3, zeta=l)
    skel.check_status(st)
    want = sketch.sparse_sign_sketch(A, l, l, 3)
    got = X.cpu().numpy() * np.sqrt(l)
    assert np.max(np.abs(got - np.round(got))) < 1e-9
    assert np.array_equal(np.round(got), np.round(want * np.sqrt(l)))
    # zeta < l: single column of A with one nonzero per row isolates each Gamma column
    m2, l2, z2 = 40, 16, 5
    A2 = np.asfortranarray(np.eye(m2))
    X2, st = skel.sketch(torch.from_numpy(A2).to(dev), l2, kind="sparse_sign", prec="f64", seed=9, zeta=z2)
    skel.check_status(st)
    assert np.array_equal(X2.cpu().numpy(), embedding.sparse_sign_embedding(l2, m2, z2, 9))


def test_sparse_sign_csc(skel, dev):
    A = workloads.snn_csc(3000, 400, 30, seed=4, density=0.08)
    l, zeta = 64, 8
    Ad = A.astype(np.float64)
    col_ptr = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    row_idx = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data.astype(np.float32)).to(dev)
    X, st = skel.sketch_csc(col_ptr, row_idx, val, A.shape[0], A.shape[1], l, seed=21, zeta=zeta)
    skel.check_status(st)
    want = sketch.sparse_sign_sketch(Ad, l, zeta, 21)
    Gam = embedding.sparse_sign_embedding(l, A.shape[0], zeta, 21)
    bound = A.shape[0] * 2.0 ** -23 * (np.abs(Gam) @ np.abs(Ad.toarray())) + 1e-300
    assert np.all(np.abs(X.cpu().numpy() - want) <= bound)


def test_gaussian_csc(skel, dev):
    A = workloads.snn_csc(500, 120, 10, seed=8, density=0.2)
    l = 24
    col_ptr = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    row_idx = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data.astype(np.float32)).to(dev)
    X, st = skel.sketch_csc(col_ptr, row_idx, val, A.shape[0], A.shape[1], l, kind="gaussian", seed=2)
    skel.check_status(st)
    Ad = A.toarray().astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 2)
    assert np.all(np.abs(X.cpu().numpy() - want) <= _bound(l, 500, 2, Ad, 2.0 ** -22) + 1e-6 * _bound(l, 500, 2, Ad, 1.0) / 500)


# column tiles of 512: 2 and 10 (clusters of 2), 3 (no cluster), 4 and 8 (clusters of 4, ragged
# last tile for n = 4000)
@pytest.mark.parametrize("m,n,l", [(1000, 777, 61), (2048, 1536, 272), (4096, 600, 130), (300, 5000, 40),
                                   (129, 513, 128), (8192, 1024, 528), (1000, 2048, 100), (600, 4000, 50)])
def test_sketch_tf32_tensor_cores(skel, dev, m, n, l):
    """tcgen05 kind::tf32 sketch: Gamma is rounded to TF32 in the kernel and A is read by the
    tensor core as TF32 (at most 2^-10 relative per operand); accumulation is FP32.  Bound:
    |dX| <= (2^-9 + m 2^-23) (|G| |A|) / sqrt(l) elementwise against the exact FP64 sketch."""
    A = workloads.dense_harmonic(m, n, seed=m + l)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="tf32", seed=77)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 77)
    G = embedding.gaussian_normals(l, m, 77)
    bound = (2.0 ** -9 + m * 2.0 ** -23) * (np.abs(G) @ np.abs(Ad)) / np.sqrt(l)
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= bound), (err / bound).max()


def test_sketch_tf32_padded_lda(skel, dev):
    """A stored with lda > m (a multiple of 4): only the m x n view is read."""
    m, n, l = 700, 300, 50
    full = np.asfortranarray(np.random.default_rng(1).standard_normal((704, n)).astype(np.float32))
    At = torch.from_numpy(full).to(dev)[:m, :]
    X, st = skel.sketch(At, l, prec="tf32", seed=3)
    skel.check_status(st)
    Ad = full[:m].astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 3)
    G = embedding.gaussian_normals(l, m, 3)
    bound = (2.0 ** -9 + m * 2.0 ** -23) * (np.abs(G) @ np.abs(Ad)) / np.sqrt(l)
    assert np.all(np.abs(X.cpu().numpy() - want) <= bound)


@pytest.mark.parametrize("m,n,l", [(1000, 777, 61), (2048, 1536, 272), (129, 513, 128), (1000, 2048, 100),
                                   (600, 4000, 50), (4100, 2048, 300)])
def test_sketch_bf16_tensor_cores(skel, dev, m, n, l):
    """tcgen05 kind::f16 sketch: the kernel rounds Gamma (evaluated in FP32) and A to BF16 to
    nearest-even; products are exact in FP32 and accumulation is FP32.  Reference: the oracle's
    BF16-operand sketch (FP64 normals rounded to BF16).  The two Gammas differ by one BF16 ulp
    (2^-7 relative) where the FP32 normal sits within a few FP32 ulps of a BF16 rounding
    boundary (about 1 entry in 10^4); at most two such entries per row are allowed for."""
    A = workloads.dense_harmonic(m, n, seed=m + l + 1)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="bf16", seed=78)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 78, operand_rounding="bf16")
    Gb = embedding.round_bf16(embedding.gaussian_normals(l, m, 78))
    Ab = embedding.round_bf16(Ad)
    acc = m * 2.0 ** -23 * (np.abs(Gb) @ np.abs(Ab))
    flips = 2 * 2.0 ** -7 * np.outer(np.abs(Gb).max(axis=1), np.abs(Ab).max(axis=0))
    bound = (acc + flips) / np.sqrt(l)
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= bound), (err / bound).max()
    # and the reduced-precision sketch stays within the BF16 operand error of the exact one
    exact = sketch.gaussian_sketch(Ad, l, 78)
    G = embedding.gaussian_normals(l, m, 78)
    assert np.all(np.abs(X.cpu().numpy() - exact) <= (2.0 ** -7 + m * 2.0 ** -23) * (np.abs(G) @ np.abs(Ad)) / np.sqrt(l))


def test_sketch_bf16_pivots_well_separated(skel, dev):
    """Pivots from the BF16 sketch equal the oracle's on columns with geometrically separated
    norms (every greedy gap far above the BF16 sketch error)."""
    rng = np.random.default_rng(10)
    m, n, k = 1500, 2048, 12
    A = rng.standard_normal((m, n)) * 1e-3
    cols = rng.choice(n, k, replace=False)
    for t, c in enumerate(cols):
        A[:, c] = rng.standard_normal(m) * 4.0 ** (k - t)
    A = np.asfortranarray(A.astype(np.float32))
    X, st = skel.sketch(torch.from_numpy(A).to(dev), k + 4, prec="bf16", seed=4)
    skel.check_status(st)
    Js, _, _, st2 = skel.pivot_lupp(X, k)
    skel.check_status(st2)
    ref = pivoting.lupp_columns(sketch.gaussian_sketch(A.astype(np.float64), k + 4, 4), k)
    assert ref["gaps"].min() > 0.2          # every step's relative gap far above BF16 rounding
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])


@pytest.mark.parametrize("prec,kind", [("f64", "gaussian"), ("f32", "gaussian"), ("tf32", "gaussian"),
                                       ("bf16", "gaussian"), ("f32", "sparse_sign"), ("f64", "sparse_sign")])
def test_sketch_row_blocks_sum_to_the_sketch(skel, dev, prec, kind):
    """The partial sketches of a row partition (row0 = multiples of 32, as dist.row_partition
    makes them for three ranks) sum to the sketch of the whole matrix: same Gamma columns,
    only the accumulation order differs."""
    from paper_2104_05877_gb300 import dist
    m, n, l = 1000, 600, 48
    dt = np.float64 if prec == "f64" else np.float32
    A = np.asfortranarray(np.random.default_rng(7).standard_normal((m, n)).astype(dt))
    At = torch.from_numpy(A).to(dev)
    X, st = skel.sketch(At, l, kind=kind, prec=prec, seed=21, zeta=6)
    skel.check_status(st)
    total = torch.zeros_like(X)
    for row0, rows in dist.row_partition(m, 3, 32):
        Xp, stp = skel.sketch(At[row0:row0 + rows], l, kind=kind, prec=prec, seed=21, zeta=6, row0=row0)
        skel.check_status(stp)
        total += Xp
    Ad = A.astype(np.float64)
    if kind == "gaussian":
        want = sketch.gaussian_sketch(Ad, l, 21)
        mag = (np.abs(embedding.gaussian_normals(l, m, 21)) @ np.abs(Ad)) / np.sqrt(l)
    else:
        want = sketch.sparse_sign_sketch(Ad, l, 6, 21)
        mag = np.abs(embedding.sparse_sign_embedding(l, m, 6, 21)) @ np.abs(Ad)
    u = 2.0 ** -52 if prec == "f64" else 2.0 ** -23
    got = total.cpu().numpy()
    assert np.all(np.abs(got - X.cpu().numpy()) <= 4 * m * u * mag)
    # and the summed partial sketch still meets the whole sketch's parity bound
    op = {"f64": 0.0, "f32": 0.0, "tf32": 2.0 ** -9, "bf16": 2.0 ** -7}[prec]
    assert np.all(np.abs(got - want) <= (op + 4 * m * u) * mag)


@pytest.mark.parametrize("prec,q,m,n", [("f64", 1, 700, 500), ("f64", 2, 700, 500), ("f32", 1, 700, 500),
                                         ("tf32", 1, 700, 500), ("tf32", 2, 700, 500), ("tf32", 1, 701, 499),
                                         ("tf32", 2, 4100, 2050)])
def test_sketch_power_iteration(skel, dev, prec, q, m, n):
    """X = Omega (A^T A)^q (Rand-LUPP-1piter for q = 1) against the oracle's definition: FP64
    to rounding; FP32 (SIMT) to FP32 accuracy; TF32 takes Omega A^T from the TF32 sketch kernel
    on a transposed copy of A (TF32 operands, 2^-10 relative each, errors of random sign:
    about 2^-11 of the norm) and the later products by 3xTF32, so it is held to 4e-3 per
    iteration -- the sketch's own precision, which is all pivot selection uses."""
    l = 40
    dt = np.float64 if prec == "f64" else np.float32
    A = workloads.dense_harmonic(m, n, seed=31, dtype=dt)
    X, st = skel.sketch_power(torch.from_numpy(A).to(dev), l, q=q, prec=prec, seed=17)
    skel.check_status(st)
    want = sketch.gaussian_sketch_power(A.astype(np.float64), l, 17, q)
    rel = np.linalg.norm(X.cpu().numpy() - want) / np.linalg.norm(want)
    assert rel <= {"f64": 1e-12, "f32": 2e-5 * q, "tf32": 4e-3 * q}[prec], rel


@pytest.mark.parametrize("m,n,l", [(1000, 777, 61), (2048, 1536, 272), (300, 129, 40), (4100, 600, 130),
                                   (129, 2048, 128)])
def test_sketch_fp8_tensor_cores(skel, dev, m, n, l):
    """tcgen05 kind::f8f6f4 sketch: e4m3 normals, A in e4m3 with one power-of-two scale per
    column, exact products, FP32 accumulation.  Reference: the oracle's FP8
    sketch (FP64 normals rounded to e4m3, the same scales).  An FP32 normal near an e4m3
    rounding boundary can round one e4m3 step (2^-3 relative) away from the FP64 one; two
    such entries per row are allowed for."""
    A = workloads.dense_harmonic(m, n, seed=m + 2 * l, dtype=np.float32)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="fp8", seed=79)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 79, operand_rounding="fp8")
    G8 = embedding.round_e4m3(embedding.gaussian_normals(l, m, 79))
    A8 = embedding.round_fp8_blocks(Ad, Ad.shape[0])
    acc = 2 * m * 2.0 ** -23 * (np.abs(G8) @ np.abs(A8))
    flips = 2 * 2.0 ** -3 * np.outer(np.abs(G8).max(axis=1), np.abs(A8).max(axis=0))
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= (acc + flips) / np.sqrt(l)), (err / ((acc + flips) / np.sqrt(l))).max()


@pytest.mark.parametrize("m,n,l", [(16384, 40, 32), (16385, 40, 32), (40000, 37, 61), (131072, 9, 16),
                                   (140000, 9, 16)])
def test_sketch_fp8_tall_columns(skel, dev, m, n, l):
    """Columns taller than one CTA's share of the quantisation (16384 rows): column j is 8 times
    larger in the 16384-row block j mod b (b blocks), so its amax and scale come from a
    different block for each j, and a block quantised with its own amax instead of the
    column's would be off by a factor near 8.  m = 16384 and 16385 straddle one block,
    131072 is the tallest clustered column (8 blocks), 140000 the two-pass path for taller
    ones.  Same bound as the FP8 test above."""
    A = workloads.dense_harmonic(m, n, seed=m % 1000 + l, dtype=np.float32)
    b = (m + 16383) // 16384
    for j in range(n):
        q = j % b
        A[q * 16384:(q + 1) * 16384, j] *= 8.0
    A = np.asfortranarray(A)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec="fp8", seed=83)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 83, operand_rounding="fp8")
    G8 = embedding.round_e4m3(embedding.gaussian_normals(l, m, 83))
    A8 = embedding.round_fp8_blocks(Ad, Ad.shape[0])
    acc = 2 * m * 2.0 ** -23 * (np.abs(G8) @ np.abs(A8))
    flips = 2 * 2.0 ** -3 * np.outer(np.abs(G8).max(axis=1), np.abs(A8).max(axis=0))
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= (acc + flips) / np.sqrt(l)), (err / ((acc + flips) / np.sqrt(l))).max()


def test_sketch_fp8_pivots_well_separated(skel, dev):
    """Pivots from the FP8 sketch equal the oracle's on its FP8 sketch (and on the exact one) for
    columns with geometrically separated norms: every greedy gap (>= 0.35 here) is far above
    the e4m3 rounding of the sketch."""
    rng = np.random.default_rng(12)
    m, n, k = 1500, 2048, 12
    A = rng.standard_normal((m, n)) * 1e-3
    cols = rng.choice(n, k, replace=False)
    for t, c in enumerate(cols):
        A[:, c] = rng.standard_normal(m) * 4.0 ** (k - t)
    A = np.asfortranarray(A.astype(np.float32))
    X, st = skel.sketch(torch.from_numpy(A).to(dev), k + 4, prec="fp8", seed=4)
    skel.check_status(st)
    Js, _, _, st2 = skel.pivot_lupp(X, k, factors=False)
    skel.check_status(st2)
    ref = pivoting.lupp_columns(sketch.gaussian_sketch(A.astype(np.float64), k + 4, 4, operand_rounding="fp8"), k)
    assert ref["gaps"].min() > 0.35
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(ref["Js"], pivoting.lupp_columns(sketch.gaussian_sketch(A.astype(np.float64), k + 4, 4), k)["Js"])
