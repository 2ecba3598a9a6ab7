"""GPU parity at full size, in the precision and launch configuration bench.py times.

8192 x 8192 FP32 (k = 256, l = 272, TF32 sketch): the oracle runs the whole path in
FP64 on the same A (a few seconds on the host): the device's sketch against the oracle's
elementwise on samples (TF32 bound), the device's pivots against the oracle's LUPP of the
device's sketch before the first near-tie at FP32 level, and the residual ||A - C Z_gpu||_F of
the device's Z formed on the host within 1.05x of the FP64 oracle's.

262144 x 4096 SNN-style CSC (~1% dense, k = 256, l = 512, sparse sign with zeta = 8):
the oracle runs end to end on the same FP32 values with scipy sparse products: the device's
sketch elementwise, its pivots before the first near-tie, and the CUR error within 1.05x.

65536 x 32768 FP32 (k = 1024, l = 1100): too large for the oracle end to end, so the
checks are ones that hold at any size: sampled sketch entries computed one by one by the
oracle, the LUPP factor's structure (|R| <= 1, R(t, j_t) = 1, X(0:s, J) = L R(:, J)), the first
two greedy pivots recomputed on the host from the device's sketch, Theorem 1's bound with the
device's eta and an independently computed rangefinder error, and the ID error of the device's Z
(the residual formed on the device) against the closed-form best rank-k error of the
constructed spectrum and within 1.05x of the FP64 GPU form's skeleton (the equal-error gate).
The FP8 sketch, bench.py's default, gets the same sampled-entry check against the oracle's FP8
sketch and the same equal-error gate.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import decomp, embedding, errors, pivoting, sketch
import workloads

pytestmark = pytest.mark.gpu


def _rel_id(sq):
    sq = sq.cpu().numpy()
    return float(np.sqrt(max(sq[0] - sq[1], 0.0) / sq[0]))


def test_dense_8192_full_size_against_oracle(skel, dev):
    m = n = 8192
    k, p = 256, 16
    l = k + p
    seed_A, seed_G = workloads.seed_for("dense_8192x8192"), workloads.seed_for("dense_8192x8192", "gamma")
    A = workloads.torch_dense_spectrum(m, n, workloads.sigma_harmonic(n), 1e-6 / np.sqrt(m), seed_A, dev,
                                       torch.float32)
    st = skel.new_status(dev)
    X, _ = skel.sketch(A, l, prec="tf32", seed=seed_G, status=st)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
    Z, sq, _ = skel.column_id(A, Js, status=st)
    e_dev, _ = skel.error(A, Js, Z=Z, status=st)
    torch.cuda.synchronize()
    skel.check_status(st)
    Ah = A.cpu().double().numpy()
    G = embedding.gaussian_normals(l, m, seed_G)
    Xo = (G @ Ah) / np.sqrt(l)
    Xg = X.cpu().double().numpy()
    # sketch: the TF32 bound on 4096 sampled entries
    rng = np.random.default_rng(0)
    ii, jj = rng.integers(0, l, 4096), rng.integers(0, n, 4096)
    mag = np.einsum("sk,ks->s", np.abs(G[ii]), np.abs(Ah[:, jj])) / np.sqrt(l)
    assert np.all(np.abs(Xg[ii, jj] - Xo[ii, jj]) <= (2.0 ** -9 + m * 2.0 ** -23) * mag)
    # pivots: the oracle's LUPP on the device's own sketch (FP64), equal before the first
    # relative gap below 1e3 FP32 roundings (the TF32 sketch itself moves X by ~1e-3, which
    # the ID-error comparison below covers)
    ref = pivoting.lupp_columns(Xg, k)
    small = np.flatnonzero(ref["gaps"] < 1e3 * 2.0 ** -23)
    pre = int(small[0]) if small.size else k
    assert pre >= 16
    assert np.array_equal(Js.cpu().numpy()[:pre], ref["Js"][:pre])
    # the device's Z: ||A - C Z_gpu||_F formed on the host in FP64, equal to the device's direct
    # residual, and within 1.05x of the FP64 oracle's ID error (its own sketch and pivots, its
    # own Z, the residual formed directly)
    J = Js.cpu().numpy()
    e_host = errors.rel_id_error(Ah, J, Z.cpu().numpy())
    e_dev = e_dev.cpu().numpy()
    assert abs(float(e_dev[1] / e_dev[0]) - e_host) <= 1e-4 * e_host
    Jo = pivoting.lupp_columns(Xo, k)["Js"]
    e_or = errors.rel_id_error(Ah, Jo, decomp.column_id(Ah, Jo))
    assert e_host <= 1.05 * e_or, (e_host, e_or)


def test_dense_65536x32768_full_size_properties(skel, dev):
    m, n = 65536, 32768
    k, p = 1024, 76
    l = k + p
    r_eff = 3300                       # exp(-3300/200) < 1e-7: the spectrum below is the floor
    seed_A, seed_G = workloads.seed_for("dense_65536x32768"), workloads.seed_for("dense_65536x32768", "gamma")
    sig = workloads.sigma_exp200(r_eff)
    g = torch.Generator(device=dev)
    g.manual_seed(seed_A)
    with torch.no_grad():
        U, _ = torch.linalg.qr(torch.randn(m, r_eff, generator=g, device=dev))
        V, _ = torch.linalg.qr(torch.randn(n, r_eff, generator=g, device=dev))
        At = V @ (U * torch.as_tensor(sig, device=dev, dtype=torch.float32)[None, :]).T   # n x m
        del U, V
        At += (1e-7 / np.sqrt(m)) * torch.randn(n, m, generator=g, device=dev)
        A = At.t()                      # m x n column-major, FP32 (built in FP32 on the device)
    st = skel.new_status(dev)
    X, _ = skel.sketch(A, l, prec="tf32", seed=seed_G, status=st)
    Js, L, R, _ = skel.pivot_lupp(X, k, factors=True, status=st)
    Z, sq, _ = skel.column_id(A, Js, status=st)
    e_dir, _ = skel.error(A, Js, Z=Z, status=st)        # ||A - C Z_gpu||_F formed on the device
    del Z
    torch.cuda.synchronize()
    skel.check_status(st)
    e_dir = e_dir.cpu().numpy()
    rel_direct = float(e_dir[1] / e_dir[0])
    # sketch entries, one by one
    rng = np.random.default_rng(1)
    ii = np.sort(rng.choice(l, 6, replace=False))
    Gi = embedding.gaussian_normals_rows(ii, m, seed_G)
    Xc = X.cpu()
    for j in rng.integers(0, n, 24):
        a = A[:, j].double().cpu().numpy()
        want = Gi @ a / np.sqrt(l)
        mag = np.abs(Gi) @ np.abs(a) / np.sqrt(l)
        got = Xc[ii, j].double().numpy()
        assert np.all(np.abs(got - want) <= (2.0 ** -9 + m * 2.0 ** -23) * mag)
    # LUPP factor structure
    J = Js.cpu().numpy()
    assert len(set(J.tolist())) == k and J.min() >= 0 and J.max() < n
    Rh = R.cpu().double().numpy()
    assert np.abs(Rh).max() <= 1.0 + 1e-6
    assert np.all(Rh[np.arange(k), J] == 1.0)
    Xs = Xc[:k].double().numpy()
    Lh = L.cpu().double().numpy()
    assert np.linalg.norm(Xs[:, J] - Lh @ Rh[:, J]) <= 1e-4 * np.linalg.norm(Xs[:, J])
    # the first two greedy pivots, recomputed from the device's sketch
    x0 = Xc[0].double().numpy()
    assert J[0] == int(np.argmax(np.abs(x0)))
    s1 = Xc[1].double().numpy() - (Xc[1, J[0]].item() / x0[J[0]]) * x0
    s1[J[0]] = 0.0
    top = np.sort(np.abs(s1))[-2:]
    if (top[1] - top[0]) / top[1] > 1e-4:
        assert J[1] == int(np.argmax(np.abs(s1)))
    # Theorem 1: ||A - C C^+ A||_F <= eta ||A - A Xt^+ Xt||_F with Xt = R (the same row space
    # as X(0:k, :)); eta from the device (skel_error), the rangefinder error from an
    # orthonormal basis of R's rows (torch QR in FP64, A Q in FP32 without TF32)
    e, st2 = skel.error(A, Js, Rf=R)
    skel.check_status(st2)
    eta = float(e[3])
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        Q, _ = torch.linalg.qr(R.t().double())
        AQ = A @ Q.float()
        nA2 = float(e[0]) ** 2
        e_rf = np.sqrt(max(nA2 - float((AQ.double() ** 2).sum()), 0.0))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    e_abs = float(e_dir[1])
    assert e_abs <= 1.05 * eta * e_rf, (e_abs, eta, e_rf)
    # the direct residual agrees with the Gram identity (which magnifies the FP32 bias of
    # ||W||^2 at this rank), and the ID error is within a small
    # factor of the best rank-k error (closed form of the constructed spectrum)
    assert abs(rel_direct - _rel_id(sq)) <= 0.1 * rel_direct       # 3.3% apart measured
    tail = np.sum(sig[k:] ** 2) + (1e-7) ** 2 * n
    best = np.sqrt(tail / (np.sum(sig ** 2) + (1e-7) ** 2 * n))
    assert rel_direct <= 5.0 * best, (rel_direct, best)
    # equal ID error: the plain FP64 GPU form (FP64 sketch and LUPP on the FP64 copy of A, the
    # path that matches the oracle bit for bit at smaller sizes) gives the reference skeleton;
    # both skeletons' IDs are formed the same way and their residuals on the device
    A64 = A.double().t().contiguous().t()
    X64, _ = skel.sketch(A64, l, prec="f64", seed=seed_G, status=st)
    J64, _, _, _ = skel.pivot_lupp(X64, k, factors=False, status=st)
    del A64, X64
    Z64, _, _ = skel.column_id(A, J64, status=st)
    e64, _ = skel.error(A, J64, Z=Z64, status=st)
    skel.check_status(st)
    e64 = e64.cpu().numpy()
    assert rel_direct <= 1.05 * float(e64[1] / e64[0]), (rel_direct, float(e64[1] / e64[0]))


def test_dense_65536x32768_fp8_sketch(skel, dev):
    """The FP8 sketch bench.py times by default, at 65536 x 32768 on the bench's A and seeds:
    sampled entries one by one against the oracle's FP8 sketch (e4m3 normals; each column of A
    in e4m3 with its power-of-two scale), with the bound of the smaller FP8 tests, and the
    equal-error gate: the ID error of the FP8 skeleton (residual formed on the device) within
    1.05x of the FP64 GPU skeleton's."""
    m, n = 65536, 32768
    k, p = 1024, 76
    l = k + p
    seed_G = workloads.seed_for("dense_65536x32768", "gamma")
    A = workloads.torch_dense_exp200(dev, m, n, seed=workloads.seed_for("dense_65536x32768"))
    st = skel.new_status(dev)
    X, _ = skel.sketch(A, l, prec="fp8", seed=seed_G, status=st)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
    Z, _, _ = skel.column_id(A, Js, status=st)
    e8, _ = skel.error(A, Js, Z=Z, status=st)
    del Z
    torch.cuda.synchronize()
    skel.check_status(st)
    rng = np.random.default_rng(2)
    ii = np.sort(rng.choice(l, 6, replace=False))
    G8 = embedding.round_e4m3(embedding.gaussian_normals_rows(ii, m, seed_G))
    Xc = X.cpu()
    for j in rng.integers(0, n, 24):
        a = A[:, j].double().cpu().numpy()
        a8 = embedding.round_fp8_blocks(a[:, None], m)[:, 0]
        want = G8 @ a8 / np.sqrt(l)
        acc = 2 * m * 2.0 ** -23 * (np.abs(G8) @ np.abs(a8))
        flips = 2 * 2.0 ** -3 * np.abs(G8).max(axis=1) * np.abs(a8).max()
        got = Xc[ii, j].double().numpy()
        assert np.all(np.abs(got - want) <= (acc + flips) / np.sqrt(l)), j
    J = Js.cpu().numpy()
    assert len(set(J.tolist())) == k and J.min() >= 0 and J.max() < n
    e8 = e8.cpu().numpy()
    rel8 = float(e8[1] / e8[0])
    A64 = A.double().t().contiguous().t()
    X64, _ = skel.sketch(A64, l, prec="f64", seed=seed_G, status=st)
    J64, _, _, _ = skel.pivot_lupp(X64, k, factors=False, status=st)
    del A64, X64
    Z64, _, _ = skel.column_id(A, J64, status=st)
    e64, _ = skel.error(A, J64, Z=Z64, status=st)
    skel.check_status(st)
    e64 = e64.cpu().numpy()
    assert rel8 <= 1.05 * float(e64[1] / e64[0]), (rel8, float(e64[1] / e64[0]))


def test_snn_262144x4096_sparse_sign_and_cur(skel, dev):
    m, n, r = 262144, 4096, 300
    k, l, zeta = 256, 512, 8
    seed_G = workloads.seed_for("snn_262144x4096", "gamma")
    A = workloads.snn_csc(m, n, r, seed=workloads.seed_for("snn_262144x4096"))          # FP32 CSC, ~1% dense
    col_ptr = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    row_idx = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data.astype(np.float32)).to(dev)
    X, st = skel.sketch_csc(col_ptr, row_idx, val, m, n, l, seed=seed_G, zeta=zeta)
    Js, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
    torch.cuda.synchronize()
    skel.check_status(st)
    A64 = A.astype(np.float64)
    # the sketch: A >= 0, so |Gamma| |A| is the sketch with every sign +; FP32 accumulation of
    # at most nnz(A(:, j)) terms in any order bounds each entry of column j
    Xo = sketch.sparse_sign_sketch(A64, l, zeta, seed_G)
    rows, _ = embedding.sparse_sign_pattern(l, m, zeta, seed_G)
    Gabs = sp.csr_matrix((np.full(m * zeta, 1.0 / np.sqrt(zeta)), (rows.ravel(), np.repeat(np.arange(m), zeta))),
                         shape=(l, m))
    mag = np.asarray((Gabs @ A64).todense())
    Xg = X.cpu().double().numpy()
    nnz_col = np.diff(A.indptr).astype(np.float64)
    assert np.all(np.abs(Xg - Xo) <= (nnz_col[None, :] + 1) * 2.0 ** -23 * mag + 1e-30)
    # pivots: the oracle's LUPP on the device's sketch, equal before the first relative gap
    # below 1e3 FP32 roundings
    ref = pivoting.lupp_columns(Xg, k)
    small = np.flatnonzero(ref["gaps"] < 1e3 * 2.0 ** -23)
    pre = int(small[0]) if small.size else k
    assert pre >= 16
    J = Js.cpu().numpy()
    assert np.array_equal(J[:pre], ref["Js"][:pre])
    # CUR on the densified A (column-major FP32 on the device): rows by LUPP on C, stable U
    cols = torch.repeat_interleave(torch.arange(n, device=dev), col_ptr[1:] - col_ptr[:-1])
    At = torch.zeros(n, m, dtype=torch.float32, device=dev)
    At[cols, row_idx.long()] = val
    Ad = At.t()
    Is, U, _, st = skel.cur(Ad, Js)
    e, _ = skel.error(Ad, Js, Is=Is, U=U, status=st)
    skel.check_status(st)
    e = e.cpu().numpy()
    e_gpu = float(e[2] / e[0])
    # the oracle end to end: its own sketch and pivots, rows by LUPP on C, stable CUR
    Jo = pivoting.lupp_columns(Xo, k)["Js"]
    Io = pivoting.lupp_rows(A64[:, Jo].toarray(), k)["Js"]
    e_or = errors.rel_cur_error(A64, Jo, decomp.cur(A64, Jo, Io), Io)
    assert e_gpu <= 1.05 * e_or, (e_gpu, e_or)

