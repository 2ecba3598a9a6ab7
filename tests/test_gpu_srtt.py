"""GPU: the SRTT sketch X = Gamma A (Sec. 2.3, item 2) against the oracle, which applies the
transform in the printed order (permute, flip signs, Hartley transform by FFT, select, scale)
and shares no arithmetic with the kernels' entry-by-entry Gamma."""
import numpy as np
import pytest
import torch

from oracle import embedding, pivoting, skeleton, sketch
import workloads

pytestmark = pytest.mark.gpu


def _mags(A, l, seed):
    """(|Gamma| |A|, the FFT's normwise term, the FP32 entry term) for the bounds below.
    Gamma's FP32 entries carry an absolute error below 2^-19 / sqrt(l) (the angle 2x/m is
    rounded before sincospif, |d cas / d angle| <= pi sqrt 2), and the oracle's FFT carries a
    normwise error ~ log2(m) u ||A(:, j)||_2 per column, times sqrt(m/l)."""
    m = A.shape[0]
    G = embedding.srtt_embedding(l, m, seed)
    mag = np.abs(G) @ np.abs(A)
    fft = 8 * np.log2(max(m, 2)) * 2.0 ** -52 * np.sqrt(m / l) * np.linalg.norm(A, axis=0)[None, :]
    ent = 2.0 ** -19 / np.sqrt(l) * np.abs(A).sum(axis=0)[None, :]
    return mag, fft, ent


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1000, 777, 61), (129, 1, 5), (64, 300, 64), (5, 7, 5)])
def test_srtt_fp64(skel, dev, m, n, l):
    A = np.asfortranarray(np.random.default_rng(m + n).standard_normal((m, n)))
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, kind="srtt", prec="f64", seed=42)
    skel.check_status(st)
    want = sketch.srtt_sketch(A, l, 42)
    mag, fft, _ = _mags(A, l, 42)
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= (m + 16) * 2.0 ** -52 * mag + fft + 1e-300), (err / ((m + 16) * 2.0 ** -52 * mag + fft)).max()
    if l == m:      # Gamma orthogonal: column norms preserved
        assert np.allclose(np.linalg.norm(X.cpu().numpy(), axis=0), np.linalg.norm(A, axis=0), rtol=1e-12)


@pytest.mark.parametrize("m,n,l", [(512, 300, 40), (1000, 130, 80), (333, 50, 333)])
def test_srtt_fp32(skel, dev, m, n, l):
    A = workloads.dense_harmonic(m, n, seed=3)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, kind="srtt", prec="f32", seed=5)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.srtt_sketch(Ad, l, 5)
    mag, fft, ent = _mags(Ad, l, 5)
    bound = (m + 8) * 2.0 ** -23 * mag + fft + ent
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("m,n,l", [(1000, 777, 61), (2048, 1536, 272), (129, 513, 128), (600, 4000, 50),
                                   (8192, 1024, 528)])
def test_srtt_tensor_cores(skel, dev, prec, m, n, l):
    """The tcgen05 sketch with Gamma's tiles generated from the SRTT tables: TF32 operands
    (2^-10 relative each) or BF16 (2^-8 each), FP32 accumulation."""
    A = workloads.dense_harmonic(m, n, seed=m + l)
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, kind="srtt", prec=prec, seed=77)
    skel.check_status(st)
    Ad = A.astype(np.float64)
    want = sketch.srtt_sketch(Ad, l, 77)
    mag, fft, ent = _mags(Ad, l, 77)
    rel = 2.0 ** -9 if prec == "tf32" else 2.0 ** -7
    bound = (rel + m * 2.0 ** -23) * mag + fft + ent
    err = np.abs(X.cpu().numpy() - want)
    assert np.all(err <= bound), (err / bound).max()


def test_srtt_full_size_sampled(skel, dev):
    """8192 x 8192 FP32, l = 272, TF32: sampled entries against rows of the oracle's Gamma."""
    m = n = 8192
    l = 272
    A = workloads.torch_dense_spectrum(m, n, workloads.sigma_harmonic(n), 1e-6 / np.sqrt(m),
                                       workloads.seed_for("dense_8192x8192"), dev, torch.float32)
    X, st = skel.sketch(A, l, kind="srtt", prec="tf32", seed=9)
    torch.cuda.synchronize()
    skel.check_status(st)
    rng = np.random.default_rng(2)
    ii = np.sort(rng.choice(l, 6, replace=False))
    Gi = embedding.srtt_embedding_rows(ii, m, l, 9)
    Xc = X.cpu()
    for j in rng.integers(0, n, 24):
        a = A[:, j].double().cpu().numpy()
        want = Gi @ a
        bound = (2.0 ** -9 + m * 2.0 ** -23) * (np.abs(Gi) @ np.abs(a)) + 2.0 ** -19 / np.sqrt(l) * np.abs(a).sum()
        assert np.all(np.abs(Xc[ii, j].double().numpy() - want) <= bound)


def test_srtt_skeleton_pivots_match_oracle(skel, dev):
    """Algorithm 2 with the SRTT sketch in FP64: the device's pivots equal the oracle's before
    the first near-tie."""
    A = workloads.dense_geometric40(600, 500, seed=8)
    k, p = 40, 10
    X, st = skel.sketch(torch.from_numpy(np.asfortranarray(A)).to(dev), k + p, kind="srtt", prec="f64", seed=3)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
    torch.cuda.synchronize()
    skel.check_status(st)
    ref = pivoting.lupp_columns(sketch.srtt_sketch(A, k + p, 3), k)
    small = np.flatnonzero(ref["gaps"] < 1e-9)
    pre = int(small[0]) if small.size else k
    assert pre >= 10
    assert np.array_equal(Js.cpu().numpy()[:pre], ref["Js"][:pre])
