"""GPU: column ID (Eq. (2.1)), stable CUR (Remark 3), errors and Theorem 1's eta."""
import numpy as np
import pytest
import torch

import oracle
from oracle import decomp, errors, pivoting, sketch
import workloads

pytestmark = pytest.mark.gpu


def _js(A, k, p, seed):
    X = sketch.gaussian_sketch(A, k + p, seed)
    return pivoting.lupp_columns(X, k)


@pytest.mark.parametrize("m,n,k", [(1000, 800, 50), (300, 200, 20), (257, 129, 1), (640, 130, 128)])
def test_id_fp64_matches_oracle(skel, dev, m, n, k):
    """FP64 mode, same J_s: ||Z_gpu - Z_or||_F <= 1e-10 ||Z_or||_F, Z(:, Js) = I."""
    A = (workloads.dense_geometric40(m, n, seed=m) if k > 1
         else np.asfortranarray(np.random.default_rng(0).standard_normal((m, n))))
    Js = _js(A, k, 10 if k + 10 <= n else 0, 1)["Js"]
    C = A[:, Js]
    kappa = np.linalg.cond(C)
    assert kappa * 2.0 ** -52 < 1e-11, f"cond(C) = {kappa:.2e} makes the 1e-10 bound unattainable"
    Z, sq, st = skel.column_id(torch.from_numpy(A).to(dev), torch.from_numpy(Js.astype(np.int32)).to(dev))
    skel.check_status(st)
    Zr = decomp.column_id(A, Js)
    Zg = Z.cpu().numpy()
    assert np.linalg.norm(Zg - Zr) <= 1e-10 * np.linalg.norm(Zr)
    assert np.max(np.abs(Zg[:, Js] - np.eye(k))) < 1e-11
    nA2, nW2 = sq.cpu().numpy()
    e2 = np.linalg.norm(A - C @ Zr) ** 2
    assert nA2 == pytest.approx(np.linalg.norm(A) ** 2, rel=1e-12)
    assert nA2 - nW2 == pytest.approx(e2, rel=1e-6, abs=1e-12 * nA2)


def test_id_fp32_error_within_gate(skel, dev):
    """FP32 QR / FP32 Q^T A / FP64 solve: the ID error stays within 1.05x of the oracle's."""
    A = workloads.dense_harmonic(2048, 1536, seed=4)
    Ad = A.astype(np.float64)
    Js = _js(Ad, 128, 16, 2)["Js"]
    Z, _, st = skel.column_id(torch.from_numpy(A).to(dev), torch.from_numpy(Js.astype(np.int32)).to(dev))
    skel.check_status(st)
    e_gpu = errors.rel_id_error(Ad, Js, Z.cpu().numpy())
    e_or = errors.rel_id_error(Ad, Js, decomp.column_id(Ad, Js))
    assert e_gpu <= 1.05 * e_or
    print(f"FP32 ID: e_gpu/e_or - 1 = {e_gpu / e_or - 1:.2e}")


def test_exact_rank_reconstruction_fp64(skel, dev):
    """Exactly rank-r input, s = r: the GPU column ID and CUR reproduce A (Lemma 1)."""
    A = workloads.exact_rank(400, 300, 12, seed=3)
    Js = _js(A, 12, 0, 5)["Js"]
    Jt = torch.from_numpy(Js.astype(np.int32)).to(dev)
    At = torch.from_numpy(A).to(dev)
    Z, _, st = skel.column_id(At, Jt)
    Is, U, _, _ = skel.cur(At, Jt, status=st)
    out, _ = skel.error(At, Jt, Z, Is, U, status=st)
    skel.check_status(st)
    e = out.cpu().numpy()
    assert e[1] / e[0] < 1e-12
    assert e[2] / e[0] < 1e-10


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_cur_matches_oracle(skel, dev, dt):
    A = workloads.dense_geometric40(600, 500, seed=8).astype(dt)
    Ad = A.astype(np.float64)
    k = 30
    Js = _js(Ad, k, 10, 3)["Js"]
    Jt = torch.from_numpy(Js.astype(np.int32)).to(dev)
    Is, U, sq, st = skel.cur(torch.from_numpy(np.asfortranarray(A)).to(dev), Jt)
    skel.check_status(st)
    Isg = Is.cpu().numpy()
    rp = pivoting.lupp_rows(Ad[:, Js], k)
    kk = int(np.argmax(rp["gaps"] < (1e-9 if dt == np.float64 else 1e-3))) if np.any(rp["gaps"] < (1e-9 if dt == np.float64 else 1e-3)) else k
    assert np.array_equal(Isg[:kk], rp["Js"][:kk])
    Ur = decomp.cur(Ad, Js, Isg)
    e_gpu = errors.rel_cur_error(Ad, Js, U.cpu().numpy(), Isg)
    e_or = errors.rel_cur_error(Ad, Js, Ur, Isg)
    assert e_gpu <= 1.05 * e_or
    if dt == np.float64:
        assert np.linalg.norm(U.cpu().numpy() - Ur) <= 1e-8 * np.linalg.norm(Ur)


@pytest.mark.parametrize("pivot", ["lupp", "cpqr"])
def test_error_and_eta_match_oracle(skel, dev, pivot):
    A = workloads.dense_harmonic(700, 500, seed=6, dtype=np.float64)
    k, l = 40, 50
    X = sketch.gaussian_sketch(A, l, 9)
    piv = pivoting.lupp_columns(X, k) if pivot == "lupp" else pivoting.cpqr_columns(X, k)
    Js = piv["Js"]
    Z = decomp.column_id(A, Js)
    Is = pivoting.lupp_rows(A[:, Js], k)["Js"]
    U = decomp.cur(A, Js, Is)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out, st = skel.error(t(np.asfortranarray(A)).t().contiguous().t(), t(Js.astype(np.int32)), t(Z),
                         t(Is.astype(np.int32)), t(U), t(piv["R"]))
    skel.check_status(st)
    e = out.cpu().numpy()
    assert e[0] == pytest.approx(np.linalg.norm(A), rel=1e-13)
    assert e[1] == pytest.approx(np.linalg.norm(A - A[:, Js] @ Z), rel=1e-10)
    assert e[2] == pytest.approx(np.linalg.norm(A - A[:, Js] @ U @ A[Is, :]), rel=1e-8)
    assert e[3] == pytest.approx(errors.eta(piv["R"], Js), rel=1e-8)
    # Theorem 1 holds with the device's numbers
    assert e[1] <= e[3] * errors.rangefinder_error(A, piv["R"]) * (1 + 1e-10)


def test_end_to_end_fp64_1000x800(skel, dev):
    """1000 x 800 FP64 (k = 50, p = 10): the whole FP64 device pipeline equals the
    oracle's skeleton, Z within 1e-10, errors within 1.05x."""
    A = workloads.dense_geometric40()
    k, p, seed = 50, 10, workloads.seed_for("dense_1000x800", "gamma")
    out = skel.skeletonize(torch.from_numpy(A).to(dev), k, p, seed=seed, prec="f64")
    torch.cuda.synchronize()
    skel.check_status(out["status"])
    ref = oracle.skeleton.skeletonize(A, k, p, seed)
    Js = out["Js"].cpu().numpy()
    small = np.flatnonzero(ref["gaps"] < 1e-9)
    kk = int(small[0]) if small.size else k
    assert np.array_equal(Js[:kk], ref["Js"][:kk])
    e = out["errors"].cpu().numpy()
    assert e[1] / e[0] <= 1.05 * ref["err_id"]
    assert e[2] / e[0] <= 1.05 * ref["err_cur"]
    if kk == k:
        assert np.linalg.norm(out["Z"].cpu().numpy() - ref["Z"]) <= 1e-10 * np.linalg.norm(ref["Z"])
        assert e[3] == pytest.approx(ref["eta"], rel=1e-8)


def test_eta_from_fp32_rfactor(skel, dev):
    """Theorem 1's eta from an FP32 R (the mixed-precision path's LUPP factor): the device's
    float-float R R^T equals the oracle's FP64 eta of the same FP32 numbers within 1e-8.
    s = 150 spans three 64-row tiles with a ragged tail; n = 3000 splits the K range."""
    rng = np.random.default_rng(31)
    m, n, k = 200, 3000, 150
    X = rng.standard_normal((m, n))
    piv = pivoting.lupp_columns(X, k)
    R32 = piv["R"].astype(np.float32)
    Js = piv["Js"]
    A = rng.standard_normal((200, n))
    out, st = skel.error(torch.from_numpy(np.asfortranarray(A)).to(dev).t().contiguous().t(),
                         torch.from_numpy(Js.astype(np.int32)).to(dev), Rf=torch.from_numpy(R32).to(dev))
    skel.check_status(st)
    assert out.cpu().numpy()[3] == pytest.approx(errors.eta(R32.astype(np.float64), Js), rel=1e-8)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_column_id_from_sketch(skel, dev, dt):
    """Z = X(:, J)^+ X over all l rows of the sketch (skel_id_sketch) against the oracle's
    least-squares solution on the same sketch: Z(:, J) = I exactly, the rest within the
    precision of the Householder QR (FP64; FP32 within 50 cond(X(:, J)) u_32); the ID from the
    sketch is never better than C^+ A."""
    A = workloads.dense_harmonic(600, 400, seed=12, dtype=np.float64)
    k, l = 30, 40
    X = sketch.gaussian_sketch(A, l, 5).astype(dt)
    Xt = torch.from_numpy(X).to(dev)
    Js, _, _, st = skel.pivot_lupp(Xt, k, factors=False)
    skel.check_status(st)
    Z, st = skel.column_id_sketch(Xt, Js)
    skel.check_status(st)
    J = Js.cpu().numpy()
    X64 = X.astype(np.float64)
    want = decomp.sketch_id(X64, J)
    got = Z.cpu().numpy()
    assert np.array_equal(got[:, J], np.eye(k))
    tol = 1e-9 if dt == np.float64 else 50 * np.linalg.cond(X64[:, J]) * 2.0 ** -24
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
    e_sk = np.linalg.norm(A - A[:, J] @ got)
    assert e_sk >= np.linalg.norm(A - A[:, J] @ decomp.column_id(A, J)) * (1 - 1e-9)


def test_mixed_path_z_accuracy(skel, dev):
    """The mixed path's Z (FP32 Householder QR, 3xTF32 W, FP64 solve) against the FP64 oracle's
    Z on the same skeleton: within a small multiple of cond(C) u_32 (stated per result; no
    FP64 refinement step)."""
    A = workloads.dense_harmonic(2048, 1500, seed=11, dtype=np.float32)
    Ad = A.astype(np.float64)
    At = torch.from_numpy(np.asfortranarray(A)).to(dev)
    X, _ = skel.sketch(At, 80, prec="tf32", seed=3)
    Js, _, _, _ = skel.pivot_lupp(X, 64, factors=False)
    Z, _, st = skel.column_id(At, Js)
    skel.check_status(st)
    J = Js.cpu().numpy()
    Zo = decomp.column_id(Ad, J)
    rel = np.linalg.norm(Z.cpu().numpy() - Zo) / np.linalg.norm(Zo)
    assert rel <= 10 * np.linalg.cond(Ad[:, J]) * 2.0 ** -24, rel


@pytest.mark.parametrize("prec,m,n", [("f64", 700, 450), ("f32", 700, 450), ("tf32", 700, 450), ("bf16", 700, 450),
                                       ("tf32", 701, 449), ("tf32", 3000, 2500)])
def test_column_sketch(skel, dev, prec, m, n):
    """Yt = Omega A^T (the column sketch of Algorithm 3) against the oracle's: SIMT FP64 / FP32
    to rounding; TF32 / BF16 by the tensor-core sketch on a transposed copy of A, within the
    operand rounding (2^-9 / 2^-7 relative per product) plus FP32 accumulation."""
    dt = np.float64 if prec == "f64" else np.float32
    A = workloads.dense_harmonic(m, n, seed=4, dtype=dt)
    Yt, st = skel.sketch_cols(torch.from_numpy(A).to(dev), 37, prec=prec, seed=9)
    skel.check_status(st)
    want = sketch.gaussian_col_sketch(A.astype(np.float64), 37, 9)
    Om = np.abs(oracle.embedding.gaussian_normals(37, n, 9)) / np.sqrt(37)
    mag = Om @ np.abs(A.astype(np.float64)).T
    u = 2.0 ** -52 if prec == "f64" else 2.0 ** -23
    op = {"f64": 0.0, "f32": 0.0, "tf32": 2.0 ** -9, "bf16": 2.0 ** -7}[prec]
    assert np.all(np.abs(Yt.cpu().numpy() - want) <= (op + 4 * n * u) * mag)


def test_streaming_skeleton_selection(skel, dev):
    """Algorithm 3 on the device (X = Gamma A, Y = A Omega^T, LUPP on X and on Y^T) against
    the oracle's: the same row and column skeletons in FP64 before the first near-tie, and a
    CUR error within 1.05x of the oracle's."""
    A = workloads.dense_harmonic(600, 500, seed=5, dtype=np.float64)
    k, p = 30, 10
    Js, Is, st = skel.skeletonize_streaming(torch.from_numpy(A).to(dev), k, p, seed=7, seed_omega=8, prec="f64")
    torch.cuda.synchronize()
    skel.check_status(st)
    ref = oracle.skeleton.streaming_skeletonize(A, k, p, 7, 8)
    for got, want, gaps in ((Js, ref["Js"], ref["gaps_x"]), (Is, ref["Is"], ref["gaps_y"])):
        small = np.flatnonzero(gaps < 1e-9)
        pre = int(small[0]) if small.size else k
        assert np.array_equal(got.cpu().numpy()[:pre], want[:pre])
    J, I = Js.cpu().numpy(), Is.cpu().numpy()
    e_gpu = errors.rel_cur_error(A, J, decomp.cur(A, J, I), I)
    assert e_gpu <= 1.05 * ref["err_cur"]


@pytest.mark.parametrize("dt,m,n,k", [(np.float64, 600, 500, 37), (np.float32, 600, 500, 37),
                                      (np.float64, 1500, 1300, 200), (np.float64, 50, 40, 1)])
def test_cur_sketch_core(skel, dev, dt, m, n, k):
    """The sketch-only CUR core U = A(Is, Js)^{-1} (Sec. 4) against the oracle's inverse, on
    the oracle's skeletons: within a condition-number multiple of the storage precision, and
    C U R reproducing A's skeleton rows and columns."""
    A = workloads.dense_harmonic(m, n, seed=3, dtype=np.float64).astype(dt)
    Ad = A.astype(np.float64)
    ref = oracle.skeleton.skeletonize(Ad, k=k, p=8, seed=4)
    Js, Is = ref["Js"], ref["Is"]
    Ur = decomp.cur_sketch(Ad, Js, Is)
    U, st = skel.cur_sketch(torch.from_numpy(np.asfortranarray(A)).to(dev),
                            torch.from_numpy(Js.astype(np.int32)).to(dev),
                            torch.from_numpy(Is.astype(np.int32)).to(dev))
    torch.cuda.synchronize()
    skel.check_status(st)
    Ug = U.cpu().numpy()
    kappa = np.linalg.cond(Ad[np.ix_(Is, Js)])
    u = 2.0 ** -52 if dt == np.float64 else 2.0 ** -23
    assert np.linalg.norm(Ug - Ur) <= 50 * k * kappa * u * np.linalg.norm(Ur)
    M = Ad[:, Js] @ Ug @ Ad[Is, :]
    assert np.linalg.norm(M[Is, :] - Ad[Is, :]) <= 50 * k * kappa * u * np.linalg.norm(Ad[Is, :])


def test_streaming_selection_tensor_cores(skel, dev):
    """Algorithm 3 with both sketches on the tensor cores (TF32): the CUR error of the
    device's skeletons within 1.05x of the FP64 oracle's."""
    A = workloads.dense_harmonic(1200, 1000, seed=5, dtype=np.float32)
    k, p = 40, 10
    Js, Is, st = skel.skeletonize_streaming(torch.from_numpy(A).to(dev), k, p, seed=7, seed_omega=8, prec="tf32")
    torch.cuda.synchronize()
    skel.check_status(st)
    Ad = A.astype(np.float64)
    ref = oracle.skeleton.streaming_skeletonize(Ad, k, p, 7, 8)
    J, I = Js.cpu().numpy(), Is.cpu().numpy()
    assert len(set(J.tolist())) == k and len(set(I.tolist())) == k
    e_gpu = errors.rel_cur_error(Ad, J, decomp.cur(Ad, J, I), I)
    assert e_gpu <= 1.05 * ref["err_cur"]


@pytest.mark.parametrize("dt,m,n,k", [(np.float64, 600, 500, 30), (np.float32, 1000, 900, 64),
                                      (np.float32, 8192, 8192, 256)])
def test_id_cur_equals_separate_calls(skel, dev, dt, m, n, k):
    """skel_id_cur (one QR of C and one W for both, the QR of R^T on the auxiliary stream)
    returns exactly what skel_id and skel_cur return separately, and the ID matches the
    oracle's."""
    if m == 8192:
        A = workloads.torch_dense_spectrum(m, n, workloads.sigma_harmonic(n), 1e-6 / np.sqrt(m),
                                           workloads.seed_for("dense_8192x8192"), dev, torch.float32)
        X, st = skel.sketch(A, k + 16, prec="tf32", seed=3)
    else:
        A = torch.from_numpy(np.asfortranarray(workloads.dense_harmonic(m, n, seed=2, dtype=dt))).to(dev)
        X, st = skel.sketch(A, k + 10, prec="f64" if dt == np.float64 else "f32", seed=3)
    Js, Is, _, _, _ = skel.pivot_skeleton(X, A, k, status=st)
    Z1, sq1, _ = skel.column_id(A, Js, status=st)
    _, U1, sqc1, _ = skel.cur(A, Js, Is, status=st)
    Z2, U2, sq2, sqc2, _ = skel.id_cur(A, Js, Is, status=st)
    torch.cuda.synchronize()
    skel.check_status(st)
    assert torch.equal(Z1, Z2) and torch.equal(U1, U2)
    assert torch.equal(sq1, sq2) and torch.equal(sqc1, sqc2)
    if m < 8192:
        Ad = A.cpu().double().numpy()
        Zr = decomp.column_id(Ad, Js.cpu().numpy())
        tol = 1e-9 if dt == np.float64 else 1e-3
        assert np.linalg.norm(Z2.cpu().numpy() - Zr) <= tol * np.linalg.norm(Zr)


@pytest.mark.parametrize("m,n,k", [(2048, 1500, 64), (4096, 4096, 256), (1001, 777, 40)])
def test_refined_z_accuracy(skel, dev, m, n, k):
    """One FP64 refinement step (skel_id_refine: corrected seminormal equations, C^T A and C^T C
    from exact FP32 products in float-float sums) takes the mixed path's Z from about
    cond(C) u_32 to within u_32 = 2^-24 of the FP64 oracle's Z on the same skeleton (relative,
    Frobenius), at least 100x closer than before; Z(:, J) = I exactly.  Measured: 7.9e-6 ->
    5.6e-9 at 4096^2, s = 256, cond(C) = 337.  (m = 1001 leaves the tensor-core W for the SIMT
    path.)"""
    A = workloads.dense_harmonic(m, n, seed=11, dtype=np.float32)
    Ad = A.astype(np.float64)
    At = torch.from_numpy(np.asfortranarray(A)).to(dev)
    X, _ = skel.sketch(At, k + 16, prec="tf32" if m % 4 == 0 else "f32", seed=3)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False)
    Z0, _, st0 = skel.column_id(At, Js)
    Z1, _, st1 = skel.column_id_refined(At, Js)
    skel.check_status(st0)
    skel.check_status(st1)
    J = Js.cpu().numpy()
    Zo = decomp.column_id(Ad, J)
    e0 = np.linalg.norm(Z0.cpu().numpy() - Zo) / np.linalg.norm(Zo)
    Z1h = Z1.cpu().numpy()
    e1 = np.linalg.norm(Z1h - Zo) / np.linalg.norm(Zo)
    assert np.array_equal(Z1h[:, J], np.eye(k))
    assert e1 <= 2.0 ** -24, (e0, e1, np.linalg.cond(Ad[:, J]))
    assert e1 <= 0.01 * e0, (e0, e1)


@pytest.mark.parametrize("m,n,k", [(2048, 1500, 64), (4096, 4096, 256)])
def test_refined_u_accuracy(skel, dev, m, n, k):
    """One FP64 refinement step of the CUR core (skel_cur_refine: the two-sided corrected
    seminormal equations, C^T A, C^T C and R R^T from exact FP32 products in float-float sums)
    takes U to within u_32 of the FP64 oracle's U on the same skeletons (relative, Frobenius),
    at least 100x closer than the unrefined mixed-path U."""
    A = workloads.dense_harmonic(m, n, seed=11, dtype=np.float32)
    Ad = A.astype(np.float64)
    At = torch.from_numpy(np.asfortranarray(A)).to(dev)
    X, _ = skel.sketch(At, k + 16, prec="tf32", seed=3)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False)
    Is, U0, _, st0 = skel.cur(At, Js)
    _, U1, _, st1 = skel.cur(At, Js, Is, refine=True)
    skel.check_status(st0)
    skel.check_status(st1)
    Uo = decomp.cur(Ad, Js.cpu().numpy(), Is.cpu().numpy())
    e0 = np.linalg.norm(U0.cpu().numpy() - Uo) / np.linalg.norm(Uo)
    e1 = np.linalg.norm(U1.cpu().numpy() - Uo) / np.linalg.norm(Uo)
    assert e1 <= 2.0 ** -24, (e0, e1)
    assert e1 <= 0.01 * e0, (e0, e1)

