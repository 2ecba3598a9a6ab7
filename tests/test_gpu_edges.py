"""GPU: degenerate shapes and inputs against the oracle: one row, one column, as many pivots
as columns, a square skeleton, blocks shorter than the sketch or narrower than k_max, and a
non-finite block in a batch."""

import numpy as np
import pytest
import torch

from oracle import decomp, pivoting, sketch, skeleton
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["tf32", "bf16", "f32"])
@pytest.mark.parametrize("m,n", [(1, 300), (200, 1), (1, 1), (33, 2)])
def test_sketch_thin_shapes(skel, dev, prec, m, n):
    rng = np.random.default_rng(m * 7 + n)
    A = np.asfortranarray(rng.standard_normal((m, n)).astype(np.float32))
    l = 20
    X, st = skel.sketch(torch.from_numpy(A).to(dev), l, prec=prec, seed=4)
    skel.check_status(st)
    want = sketch.gaussian_sketch(A.astype(np.float64), l, 4)
    G = np.abs(sketch.embedding.gaussian_normals(l, m, 4))
    op = {"tf32": 2.0 ** -9, "bf16": 2.0 ** -7, "f32": 0.0}[prec]
    bound = (op + 4 * m * 2.0 ** -23) * (G @ np.abs(A.astype(np.float64))) / np.sqrt(l) + 1e-30
    assert np.all(np.abs(X.cpu().numpy() - want) <= bound)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("l,n,s", [(40, 40, 40), (30, 25, 25), (10, 500, 1)])
def test_lupp_all_columns_and_one(skel, dev, dt, l, n, s):
    """s = n (every column pivoted, the last steps with a single candidate) and s = 1."""
    X = np.random.default_rng(l + n + s).standard_normal((l, n)).astype(dt)
    Js, L, R, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X.astype(np.float64), s)
    small = np.flatnonzero(ref["gaps"] < (1e-9 if dt == np.float64 else 1e-4))
    pre = int(small[0]) if small.size else s
    assert np.array_equal(Js.cpu().numpy()[:pre], ref["Js"][:pre])
    assert sorted(Js.cpu().numpy().tolist()) == sorted(set(Js.cpu().numpy().tolist()))


@pytest.mark.parametrize("m,s", [(48, 48), (300, 1), (64, 64)])
def test_column_id_square_and_single(skel, dev, m, s):
    """C square (s = m) and a single skeleton column."""
    A = workloads.dense_harmonic(m, 120, seed=m + s, dtype=np.float64)
    Js = np.random.default_rng(s).choice(120, s, replace=False).astype(np.int32)
    Z, sq, st = skel.column_id(torch.from_numpy(A).to(dev), torch.from_numpy(Js).to(dev))
    skel.check_status(st)
    want = decomp.column_id(A, Js)
    assert np.linalg.norm(Z.cpu().numpy() - want) <= 1e-9 * np.linalg.norm(want)


def test_cur_single_skeleton(skel, dev):
    A = workloads.dense_harmonic(200, 150, seed=3, dtype=np.float64)
    Js = torch.tensor([17], dtype=torch.int32, device=dev)
    Is, U, sq, st = skel.cur(torch.from_numpy(A).to(dev), Js)
    skel.check_status(st)
    want = decomp.cur(A, [17], Is.cpu().numpy())
    assert np.allclose(U.cpu().numpy(), want, rtol=1e-9, atol=0)


@pytest.mark.parametrize("s", [1, 60])
def test_id_sketch_one_and_all(skel, dev, s):
    """The sketch-only ID with one pivot and with as many pivots as columns (Z = I)."""
    X = np.random.default_rng(s).standard_normal((70, 60))
    Xd = torch.from_numpy(X).to(dev)
    Js, _, _, st = skel.pivot_lupp(Xd, s, factors=False)
    skel.check_status(st)
    Z, st = skel.column_id_sketch(Xd, Js)
    skel.check_status(st)
    J = Js.cpu().numpy()
    assert np.allclose(Z.cpu().numpy(), decomp.sketch_id(X, J), rtol=0, atol=1e-9)
    if s == 60:
        assert np.array_equal(Z.cpu().numpy()[:, J], np.eye(60))


def test_batch_degenerate_blocks(skel, dev):
    """A single column, a block shorter than the sketch (rank <= m_b), and k_max above n_b."""
    rng = np.random.default_rng(2)
    blocks = [rng.standard_normal((100, 1)), rng.standard_normal((5, 80)), rng.standard_normal((300, 7)),
              workloads.kernel_blocks(1, seed=3, mrange=(200, 200), nrange=(150, 150))[0].astype(np.float64)]
    tb = [torch.from_numpy(np.asfortranarray(B.astype(np.float32))).to(dev) for B in blocks]
    plan = skel.BatchPlan(tb, 16, p=8, tol=1e-6, seed=3)
    Js, ranks, Z, st = plan.run()
    torch.cuda.synchronize()
    skel.check_status(st)
    ranks = ranks.cpu().numpy()
    ref = skeleton.batch_skeletonize([B.astype(np.float32).astype(np.float64) for B in blocks], 16, 8, 1e-6, 3)
    assert ranks[0] == 1 and ranks[2] == 7
    assert ranks[1] == ref[1]["rank"] <= 5
    assert abs(int(ranks[3]) - ref[3]["rank"]) <= 1


def test_batch_nonfinite_block_reported(skel, dev):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((120, 90)).astype(np.float32)
    A[7, 3] = np.nan
    plan = skel.BatchPlan([torch.from_numpy(np.asfortranarray(A)).to(dev)], 12, p=8, tol=1e-6, seed=1)
    _, _, _, st = plan.run()
    torch.cuda.synchronize()
    assert int(st[0].item()) == 3          # SKEL_ERR_NONFINITE, and no fault or hang
