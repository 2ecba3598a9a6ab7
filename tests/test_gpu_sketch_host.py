"""GPU: the sketch of a host-resident A streamed in column panels (skel_sketch_host) against the
oracle and against the device sketch of the same A.  X's columns j0..j1 depend only on A's
columns j0..j1 (Algorithm 1, sketch step), so any panel width gives the same sketch up to the
summation order of the K-split."""
import numpy as np
import pytest
import torch

from oracle import embedding, sketch
import workloads

pytestmark = pytest.mark.gpu


def _mag(l, m, seed, Ad):
    return (np.abs(embedding.gaussian_normals(l, m, seed)) @ np.abs(Ad)) / np.sqrt(l)


@pytest.mark.parametrize("panel", [256, 0, 1300, 7])
def test_sketch_host_fp64_panels(skel, dev, panel):
    """FP64, pageable host A with lda > m (a view of a taller array): ragged last panel
    (1300 = 5 x 256 + 20), one panel (0 and 1300) and narrow odd panels (7)."""
    m, n, l = 1000, 1300, 37
    full = np.asfortranarray(np.random.default_rng(3).standard_normal((1003, n)))
    A = torch.from_numpy(full)[:m, :]
    X, st = skel.sketch_host(A, l, prec="f64", seed=42, panel=panel)
    skel.check_status(st)
    Ad = full[:m]
    want = sketch.gaussian_sketch(Ad, l, 42)
    assert np.all(np.abs(X.cpu().numpy() - want) <= m * 2.0 ** -52 * _mag(l, m, 42, Ad) + 1e-300)


@pytest.mark.parametrize("prec,m,n,l,panel", [("tf32", 1001, 2000, 61, 512), ("tf32", 4100, 3000, 272, 0),
                                              ("tf32", 2048, 1536, 130, 256), ("bf16", 1001, 2000, 61, 768),
                                              ("f32", 777, 900, 40, 300)])
def test_sketch_host_single_precision(skel, dev, prec, m, n, l, panel):
    """Pinned host A, m not a multiple of 4 (the staging columns are padded): the oracle's bound
    for the precision, and agreement with skel.sketch on the device copy."""
    A = torch.from_numpy(workloads.dense_harmonic(m, n, seed=m + l)).pin_memory()
    X, st = skel.sketch_host(A, l, prec=prec, seed=77, panel=panel)
    Xd, std = skel.sketch(A.to(dev), l, prec=prec, seed=77)
    skel.check_status(st)
    skel.check_status(std)
    Ad = A.numpy().astype(np.float64)
    want = sketch.gaussian_sketch(Ad, l, 77)
    op = {"f32": 0.0, "tf32": 2.0 ** -9, "bf16": 2.0 ** -7}[prec]
    mag = _mag(l, m, 77, Ad)
    got = X.cpu().numpy()
    assert np.all(np.abs(got - want) <= (op + 2 * m * 2.0 ** -23) * mag)
    # same operand rounding as the device path: only the accumulation order differs
    assert np.all(np.abs(got - Xd.cpu().numpy()) <= 4 * m * 2.0 ** -23 * mag)


def test_sketch_host_fp8(skel, dev):
    """FP8: the scales are per column, so a column panel scales exactly as the whole matrix
    does."""
    m, n, l = 1000, 1200, 61
    A = torch.from_numpy(workloads.dense_harmonic(m, n, seed=5, dtype=np.float32)).pin_memory()
    X, st = skel.sketch_host(A, l, prec="fp8", seed=79, panel=256)
    Xd, std = skel.sketch(A.to(dev), l, prec="fp8", seed=79)
    skel.check_status(st)
    skel.check_status(std)
    G8 = embedding.round_e4m3(embedding.gaussian_normals(l, m, 79))
    A8 = embedding.round_fp8_blocks(A.numpy().astype(np.float64), m)
    acc = 4 * m * 2.0 ** -23 * (np.abs(G8) @ np.abs(A8)) / np.sqrt(l)
    assert np.all(np.abs(X.cpu().numpy() - Xd.cpu().numpy()) <= acc)


@pytest.mark.parametrize("kind,prec", [("sparse_sign", "f64"), ("sparse_sign", "f32"), ("srtt", "f64"),
                                       ("srtt", "tf32")])
def test_sketch_host_other_embeddings(skel, dev, kind, prec):
    m, n, l = 900, 1000, 40
    dt = np.float64 if prec == "f64" else np.float32
    Ad = np.asfortranarray(np.random.default_rng(9).standard_normal((m, n)))
    A = torch.from_numpy(Ad.astype(dt))
    X, st = skel.sketch_host(A, l, kind=kind, prec=prec, seed=13, zeta=6, panel=384)
    skel.check_status(st)
    A64 = A.numpy().astype(np.float64)
    if kind == "sparse_sign":
        want = sketch.sparse_sign_sketch(A64, l, 6, 13)
        mag = np.abs(embedding.sparse_sign_embedding(l, m, 6, 13)) @ np.abs(A64)
    else:
        want = sketch.srtt_sketch(A64, l, 13)
        mag = np.abs(embedding.srtt_embedding(l, m, 13)) @ np.abs(A64)
    u = 2.0 ** -52 if prec == "f64" else 2.0 ** -23
    op = 2.0 ** -9 if prec == "tf32" else 0.0
    assert np.all(np.abs(X.cpu().numpy() - want) <= (op + 4 * m * u) * mag + 1e-300)


def test_sketch_host_edges(skel, dev):
    # n = 0: nothing to do
    X, st = skel.sketch_host(torch.zeros(10, 0, dtype=torch.float64), 3, prec="f64")
    skel.check_status(st)
    assert X.shape == (3, 0)
    # m = 0: the sketch of an empty column is zero
    X, st = skel.sketch_host(torch.zeros(0, 5, dtype=torch.float32), 4, prec="tf32")
    skel.check_status(st)
    assert torch.all(X == 0)
    # a negative panel width is an argument error
    with pytest.raises(skel.SkelError) as e:
        skel.sketch_host(torch.zeros(8, 8, dtype=torch.float64), 3, prec="f64", panel=-1)
    assert e.value.code == 1
    # non-finite data is reported on the device
    A = np.random.default_rng(0).standard_normal((50, 600))
    A[7, 530] = np.nan
    _, st = skel.sketch_host(torch.from_numpy(np.asfortranarray(A)), 8, prec="f64", panel=256)
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 3


def test_sketch_host_then_pivots(skel, dev):
    """The skeleton from the streamed sketch equals the one from the device sketch (FP64: the
    two sketches agree to rounding and the pivots' gaps are far above it)."""
    m, n, l, k = 2000, 1500, 40, 30
    A = np.asfortranarray(workloads.dense_geometric40(m, n, seed=11))
    X, st = skel.sketch_host(torch.from_numpy(A), l, prec="f64", seed=5, panel=512)
    Xd, std = skel.sketch(torch.from_numpy(A).to(dev), l, prec="f64", seed=5)
    J, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
    Jd, _, _, _ = skel.pivot_lupp(Xd, k, factors=False, status=std)
    skel.check_status(st)
    skel.check_status(std)
    assert torch.equal(J.cpu(), Jd.cpu())


def _col_mag(l, n, seed, Ad):
    return (np.abs(embedding.gaussian_normals(l, n, seed)) @ np.abs(Ad).T) / np.sqrt(l)


@pytest.mark.parametrize("prec,m,n,l,panel", [("f64", 700, 1300, 37, 256), ("f64", 700, 1301, 37, 0),
                                              ("f32", 777, 900, 40, 300), ("tf32", 1001, 2000, 61, 512),
                                              ("tf32", 2048, 1536, 130, 4), ("bf16", 1001, 1000, 61, 768)])
def test_two_sided_single_pass(skel, dev, prec, m, n, l, panel):
    """Both sketches of Algorithm 3 from one pass over a host A: X against the oracle's row
    sketch and Yt against its column sketch, each within the precision's bound, and both
    against the device calls on the same A (only the order of the sums differs; Yt adds one
    partial per panel)."""
    dt = np.float64 if prec == "f64" else np.float32
    A = np.asfortranarray(np.random.default_rng(m + n).standard_normal((m, n)).astype(dt))
    X, Yt, st = skel.sketch_host_two_sided(torch.from_numpy(A), l, prec=prec, seed=7, seed_omega=8, panel=panel)
    Ad_dev = torch.from_numpy(A).to(dev)
    Xd, _ = skel.sketch(Ad_dev, l, prec=prec, seed=7, status=st)
    Ytd, _ = skel.sketch_cols(Ad_dev, l, prec=prec, seed=8, status=st)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    u = 2.0 ** -52 if prec == "f64" else 2.0 ** -23
    op = {"f64": 0.0, "f32": 0.0, "tf32": 2.0 ** -9, "bf16": 2.0 ** -7}[prec]
    mx, my = _mag(l, m, 7, Ad), _col_mag(l, n, 8, Ad)
    gx, gy = X.cpu().numpy(), Yt.cpu().numpy()
    assert np.all(np.abs(gx - sketch.gaussian_sketch(Ad, l, 7)) <= (op + 2 * m * u) * mx + 1e-300)
    assert np.all(np.abs(gy - sketch.gaussian_col_sketch(Ad, l, 8)) <= (op + 2 * n * u) * my + 1e-300)
    assert np.all(np.abs(gx - Xd.cpu().numpy()) <= 4 * m * u * mx + 1e-300)
    assert np.all(np.abs(gy - Ytd.cpu().numpy()) <= 4 * n * u * my + 1e-300)


def test_streaming_selection_host_one_pass(skel, dev):
    """Algorithm 3 on a host A in one pass: the same row and column skeletons as the oracle's
    in FP64 before the first near-tie (the oracle forms both sketches from the whole A)."""
    from oracle import skeleton
    A = np.asfortranarray(workloads.dense_harmonic(600, 500, seed=5, dtype=np.float64))
    k, p = 30, 10
    Js, Is, st = skel.skeletonize_streaming_host(torch.from_numpy(A), k, p, seed=7, seed_omega=8, prec="f64",
                                                 panel=128)
    skel.check_status(st)
    ref = skeleton.streaming_skeletonize(A, k, p, 7, 8)
    for got, want, gaps in ((Js, ref["Js"], ref["gaps_x"]), (Is, ref["Is"], ref["gaps_y"])):
        small = np.flatnonzero(gaps < 1e-9)
        pre = int(small[0]) if small.size else k
        assert np.array_equal(got.cpu().numpy()[:pre], want[:pre])


def test_two_sided_argument_errors(skel, dev):
    A = torch.zeros(64, 64, dtype=torch.float32)
    for kw, code in (({"panel": 6}, 1), ({"panel": -4}, 1), ({"prec": "fp8"}, 7)):
        args = {"prec": "tf32", "panel": 0}
        args.update(kw)
        with pytest.raises(skel.SkelError) as e:
            skel.sketch_host_two_sided(A, 8, **args)
        assert e.value.code == code
    with pytest.raises(skel.SkelError) as e:     # FP64 arithmetic needs FP64 storage
        skel.sketch_host_two_sided(A, 8, prec="f64")
    assert e.value.code == 1
