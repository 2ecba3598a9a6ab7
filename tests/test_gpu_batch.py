"""GPU: batched skeletonization (skel_batch_*) against the oracle's per-block pipeline
(sketch with one Gamma, LUPP stopped at the tolerance rank, sketch-only column ID)."""

import numpy as np
import pytest
import torch

from oracle import skeleton
import workloads

pytestmark = pytest.mark.gpu


def _run(skel, dev, blocks, kmax, p, tol, seed):
    tb = [torch.from_numpy(np.asfortranarray(B.astype(np.float32))).to(dev) for B in blocks]
    plan = skel.BatchPlan(tb, kmax, p=p, tol=tol, seed=seed)
    Js, ranks, Z, st = plan.run()
    torch.cuda.synchronize()
    skel.check_status(st)
    return plan, Js.cpu().numpy(), ranks.cpu().numpy(), Z


def _id_error(A, Js, Z):
    A = A.astype(np.float64)
    return np.linalg.norm(A - A[:, Js] @ Z) / np.linalg.norm(A)


def _exact_rank_blocks():
    """Blocks of exact rank r_b with singular values 2^-t (t < r_b <= 18): every one is above
    tol = 1e-6 and FP32-resolvable, and nothing is left after r_b steps."""
    rng = np.random.default_rng(8)
    blocks, ranks_true = [], []
    for m, n in [(300, 100), (700, 260), (150, 400), (1000, 520), (400, 800), (64, 64)]:
        r = int(rng.integers(3, 19))
        U, _ = np.linalg.qr(rng.standard_normal((m, r)))
        V, _ = np.linalg.qr(rng.standard_normal((n, r)))
        blocks.append(((U * 2.0 ** -np.arange(r)) @ V.T).astype(np.float32).astype(np.float64))
        ranks_true.append(r)
    return blocks, ranks_true


def test_batch_exact_rank_blocks(skel, dev):
    """Exact-rank blocks: the true rank, pivots equal to the oracle's before its first relative
    gap below 1e-3, Z(:, Js) = I, rows past the rank zero, and a reconstruction to FP32 level.
    Widths cover one and two CTAs per block at this l."""
    blocks, ranks_true = _exact_rank_blocks()
    kmax, p, tol, seed = 40, 16, 1e-5, 5       # FP32 rounding of A leaves ~1e-7 after r steps
    plan, Js, ranks, Z = _run(skel, dev, blocks, kmax, p, tol, seed)
    ref = skeleton.batch_skeletonize(blocks, kmax, p, tol, seed)
    for b, A in enumerate(blocks):
        r = int(ranks[b])
        assert r == ref[b]["rank"] == ranks_true[b]
        small = np.flatnonzero(ref[b]["gaps"] < 1e-3)
        pre = int(small[0]) if small.size else r
        assert np.array_equal(Js[b, :pre], ref[b]["Js"][:pre])
        assert np.all(Js[b, r:] == -1)
        zb = plan.z_block(Z, b).cpu().numpy()
        assert np.all(zb[r:] == 0)
        assert np.array_equal(zb[:r][:, Js[b, :r]], np.eye(r))
        assert _id_error(A, Js[b, :r], zb[:r]) < 1e-5


def test_batch_kernel_blocks_config4_style(skel, dev):
    """Gaussian-kernel blocks between separated point clusters (config 4's generator, smaller
    batch): the oracle's rank, or, where its estimate is within 2x of the threshold, a rank
    within 15% of it, pivots equal before the first step whose absolute gap is within 1e3
    FP32 roundings of X, and the ID error
    within 1.05x of the oracle's plus half the tolerance (the FP32 sketch and back substitution
    leave a noise floor of that order at tol = 1e-6; 3 tol when the ranks differ)."""
    blocks = workloads.kernel_blocks(40, seed=14, mrange=(64, 1024), nrange=(64, 700))
    blocks = [B.astype(np.float64) for B in blocks]
    kmax, p, tol, seed = 128, 16, 1e-6, 9
    plan, Js, ranks, Z = _run(skel, dev, blocks, kmax, p, tol, seed)
    ref = skeleton.batch_skeletonize(blocks, kmax, p, tol, seed)
    for b, A in enumerate(blocks):
        r, ro = int(ranks[b]), ref[b]["rank"]
        est = np.array(ref[b]["estimates"]) / tol ** 2
        near = est[ro] > 0.5 or (ro > 0 and est[ro - 1] < 2.0)
        # near the threshold the decision is ill-conditioned: once the pivot paths part on a
        # tiny gap the two estimates cross it a few steps apart
        assert r == ro or (near and abs(r - ro) <= max(1, int(0.15 * ro))), (b, r, ro, est[max(ro - 1, 0):ro + 1])
        # the comparison stops at the first step whose absolute gap is within 1e3 x the FP32
        # rounding of X (the parity contract's delta, on the Schur complement's own scale)
        thr = 1e3 * 2.0 ** -23 * np.abs(ref[b]["X"]).max()
        small = np.flatnonzero(ref[b]["gaps"] * ref[b]["mags"] < thr)
        pre = min(r, ro, int(small[0]) if small.size else ro)
        assert np.array_equal(Js[b, :pre], ref[b]["Js"][:pre])
        zb = plan.z_block(Z, b, r).cpu().numpy()
        e_gpu = _id_error(A, Js[b, :r], zb)
        e_or = _id_error(A, ref[b]["Js"], ref[b]["Z"])
        # FP32 sketch and FP32 back substitution: a noise floor of a fraction of tol at this level
        assert e_gpu <= (1.05 * e_or + 0.5 * tol if r == ro else 3 * tol), (b, e_gpu, e_or)
        assert e_gpu <= 2 * tol


def test_batch_rank_capped_and_narrow_blocks(skel, dev):
    """Full-rank noise blocks stop at kmax; a block narrower than kmax stops when no column
    is left (rank = n_b)."""
    rng = np.random.default_rng(6)
    blocks = [rng.standard_normal((200, 150)), rng.standard_normal((300, 12))]
    kmax = 24
    plan, Js, ranks, Z = _run(skel, dev, blocks, kmax, 8, 1e-6, 1)
    assert ranks[0] == kmax and ranks[1] == 12
    assert sorted(Js[1, :12]) == list(range(12)) and np.all(Js[1, 12:] == -1)


def test_batch_graph_and_autotune_change_no_result(skel, dev):
    """A plan with the autotuner (sketch pipeline depth, LUPP classes serial or concurrent) and
    a captured CUDA graph returns exactly what a plain plan returns, on every replay, and
    re-captures when its outputs change; blocks of all three cluster classes are present."""
    blocks = workloads.torch_kernel_blocks(96, workloads.seed_for(4) + 7, dev)
    blocks[0] = torch.randn(900, 2000, device=dev).t().contiguous().t()[:, :1900]    # a 4-CTA block
    blocks[1] = torch.randn(800, 1000, device=dev).t().contiguous().t()               # a 2-CTA block
    kw = dict(p=16, tol=1e-6, seed=11)
    plain = skel.BatchPlan(blocks, 64, **kw)
    Js0, r0, Z0, st0 = plain.run()
    tuned = skel.BatchPlan(blocks, 64, graph=True, autotune=True, **kw)
    assert tuned.info["flags"] == 3 and tuned.info["sketch_stages"] in (2, 3)
    for _ in range(3):
        Js1, r1, Z1, st1 = tuned.run()
        torch.cuda.synchronize()
        skel.check_status(st1)
        assert torch.equal(Js0, Js1) and torch.equal(r0, r1) and torch.equal(Z0, Z1)
    st2 = skel.new_status(dev)
    Js2, r2, Z2, _ = tuned.run(status=st2)     # new outputs: captured again
    torch.cuda.synchronize()
    skel.check_status(st0)
    skel.check_status(st2)
    assert torch.equal(Js0, Js2) and torch.equal(r0, r2) and torch.equal(Z0, Z2)
