"""GPU: LUPP and CPQR on the sketch (Sec. 2.5) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import pivoting, errors, sketch
import workloads

pytestmark = pytest.mark.gpu


def _prefix(gaps, delta):
    """Number of leading steps whose oracle gap is at least delta."""
    small = np.flatnonzero(gaps < delta)
    return int(small[0]) if small.size else len(gaps)


@pytest.mark.parametrize("l,n,s", [(20, 100, 20), (60, 800, 50), (8, 8, 8), (30, 5000, 1),
                                   (128, 3001, 100), (256, 8192, 256)])
def test_lupp_fp64_bit_exact(skel, dev, l, n, s):
    """Same FP64 X in, same operation order: pivots and factors are bit-identical."""
    X = np.random.default_rng(l * n + s).standard_normal((l, n))
    Js, Lf, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X, s)
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(Rf.cpu().numpy(), ref["R"])
    assert np.array_equal(Lf.cpu().numpy(), ref["L"][:s, :s])


def test_lupp_fp64_global_slab_path(skel, dev):
    """s x (n / G) too large for shared memory: the slab lives in the global workspace."""
    l, n, s = 520, 8192, 512
    X = np.random.default_rng(3).standard_normal((l, n))
    Js, _, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X, s)
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(Rf.cpu().numpy(), ref["R"])


@pytest.mark.parametrize("l,n,s", [(80, 70000, 70), (20, 300000, 20)])
def test_lupp_fp64_grid_panels_bit_exact(skel, dev, l, n, s):
    """Too wide for a cluster panel (n / 16 columns per CTA overflow shared memory): grid-wide
    panels of b rows over every SM, the trailing rows' multipliers by forward substitution and
    the tiled trailing update.  Textbook operation order, so Js, L and R are bit-identical to
    the FP64 oracle's (70 steps: panels of 54 and 16 rows)."""
    X = np.random.default_rng(l * n + s).standard_normal((l, n))
    Js, Lf, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X, s)
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(Rf.cpu().numpy(), ref["R"])
    assert np.array_equal(Lf.cpu().numpy(), ref["L"][:s, :s])


def test_lupp_fp32_grid_panels_tall_rows(skel, dev):
    """FP32 row LUPP of a tall C (262144 x 96, as for the tall sparse configuration's CUR), on the
    grid-panel path: C = 0.01 N(0, 1) plus C(i_q, q) = 1 in distinct random rows, so step q
    picks row i_q with a wide gap; the pivots equal the FP64 oracle's and the planted rows, and
    the factor has |R| <= 1 with R(t, j_t) = 1."""
    rng = np.random.default_rng(9)
    m, s = 262144, 96
    C = 0.01 * rng.standard_normal((m, s))
    rows = rng.choice(m, s, replace=False)
    C[rows, np.arange(s)] = 1.0
    C = np.asfortranarray(C.astype(np.float32))
    Is, st = skel.pivot_lupp_rows(torch.from_numpy(C).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_rows(C.astype(np.float64), s)
    assert np.array_equal(ref["Js"], rows)
    assert np.array_equal(Is.cpu().numpy(), ref["Js"])
    Xt = torch.from_numpy(np.ascontiguousarray(C.T)).to(dev)
    Js, _, Rf, st = skel.pivot_lupp(Xt, s)
    skel.check_status(st)
    R = Rf.cpu().numpy()
    J = Js.cpu().numpy()
    assert np.array_equal(J, rows)
    assert np.abs(R).max() <= 1.0 and np.all(R[np.arange(s), J] == 1.0)


def _separated(l, n, seed, ratio):
    """Gaussian X with geometric column scales in random order: wide pivot gaps."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((l, n)) * ratio ** rng.permutation(n)[None, :]).astype(np.float32)


@pytest.mark.parametrize("l,n,s,ratio,min_prefix", [(40, 1000, 32, 0.7, 32), (300, 4096, 256, 0.93, 200),
                                                    (300, 4096, 256, 1.0, 0)])
def test_lupp_fp32_prefix(skel, dev, l, n, s, ratio, min_prefix):
    """FP32 arithmetic: pivots equal the FP64 oracle's up to the first step whose relative
    gap is below 1e-3 (1e4 x the FP32 unit roundoff); on well-separated inputs that prefix
    covers (nearly) every step."""
    X = _separated(l, n, n + s, ratio)
    Js, _, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X.astype(np.float64), s)
    k = _prefix(ref["gaps"], 1e-3)
    assert k >= min_prefix
    assert np.array_equal(Js.cpu().numpy()[:k], ref["Js"][:k])
    R = Rf.cpu().numpy()
    assert np.max(np.abs(R)) <= 1.0 + 1e-6
    assert np.allclose(R[np.arange(s), Js.cpu().numpy()], 1.0)


def test_lupp_kahan_ties(skel, dev):
    """Lemma 2's Kahan-type X: ties at every step resolve to the lowest index."""
    for dt in (torch.float64, torch.float32):
        X = workloads.kahan_type(12, 40)
        Js, _, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev, dt), 12)
        skel.check_status(st)
        assert np.array_equal(Js.cpu().numpy(), np.arange(12))
        assert np.array_equal(Rf.cpu().numpy().astype(np.float64), X)


def test_lupp_rank_deficient(skel, dev):
    X = np.zeros((4, 50))
    X[0, 7] = 2.0
    X[1, 9] = -1.0
    Js, _, _, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), 4)
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 4
    assert list(Js.cpu().numpy()) == [7, 9, -1, -1]


def test_lupp_nonfinite(skel, dev):
    X = np.random.default_rng(0).standard_normal((6, 30))
    X[0, 4] = np.inf
    _, _, _, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), 3)
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 3


@pytest.mark.parametrize("m,s", [(500, 20), (8192, 64), (20000, 129)])
def test_row_lupp_on_tall_C(skel, dev, m, s):
    """Algorithm 2, row pivoting: row pivots of C (column-major) via LUPP on C^T."""
    C = np.asfortranarray(np.random.default_rng(m).standard_normal((m, s)))
    Is, st = skel.pivot_lupp_rows(torch.from_numpy(C).to(dev), s)
    skel.check_status(st)
    assert np.array_equal(Is.cpu().numpy(), pivoting.lupp_rows(C, s)["Js"])


@pytest.mark.parametrize("l,n,s,dt,ratio,min_prefix", [(20, 300, 20, np.float64, 1.0, 2), (64, 2000, 48, np.float64, 1.0, 1),
                                                      (80, 8192, 64, np.float32, 0.95, 20), (40, 777, 30, np.float32, 0.8, 30),
                                                      (80, 8192, 64, np.float32, 1.0, 0)])
def test_cpqr_prefix(skel, dev, l, n, s, dt, ratio, min_prefix):
    X = _separated(l, n, l + n, ratio).astype(dt)
    Js, Rf, st = skel.pivot_cpqr(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.cpqr_columns(X.astype(np.float64), s)
    delta = 1e-9 if dt == np.float64 else 1e-3
    k = _prefix(ref["gaps"], delta)
    assert k >= min_prefix
    Jg = Js.cpu().numpy()
    assert np.array_equal(Jg[:k], ref["Js"][:k])
    R = Rf.cpu().numpy().astype(np.float64)
    tol = 1e-10 if dt == np.float64 else 2e-4
    assert np.allclose(np.abs(R[np.arange(k), Jg[:k]]), np.abs(ref["R"][np.arange(k), ref["Js"][:k]]), rtol=tol)
    # R(:, J) is upper triangular in pivot order and, the reflectors being orthogonal,
    # R(:, J)^T R(:, J) reproduces the Gram matrix X(:, J)^T X(:, J) of the selected columns
    R1 = R[:, Jg]
    assert np.array_equal(np.triu(R1), R1)
    XJ = X.astype(np.float64)[:, Jg]
    gram_tol = 1e-12 if dt == np.float64 else 5e-5
    assert np.linalg.norm(R1.T @ R1 - XJ.T @ XJ) <= gram_tol * np.linalg.norm(XJ) ** 2


def test_cpqr_kahan_like_separated(skel, dev):
    """Columns of strictly decreasing norm, orthogonal: CPQR picks them in norm order."""
    l, n = 16, 64
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((l, l)))
    X = np.zeros((l, n))
    perm = rng.permutation(n)
    for r in range(l):
        X[:, perm[r]] = Q[:, r] * 2.0 ** (-r)
    Js, Rf, st = skel.pivot_cpqr(torch.from_numpy(X).to(dev), l)
    skel.check_status(st)
    assert np.array_equal(Js.cpu().numpy(), perm[:l])


def test_grid_wait_times_out(skel, dev):
    """A grid-wide wait that can never complete returns SKEL_ERR_TIMEOUT after its limit and
    leaves the context usable."""
    st = skel.debug_grid_timeout(8, 200_000_000, device=dev)
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 5
    X = torch.randn(4, 40, dtype=torch.float64, device=dev)
    Js, _, _, st2 = skel.pivot_lupp(X, 4)
    skel.check_status(st2)


def test_lupp_very_wide_uses_grid_kernel(skel, dev):
    """400000 columns: a panel of even 8 rows does not fit one cluster's shared memory, so
    the grid-barrier kernel runs, with its column slab in the global workspace (FP64);
    factors stay bit-identical to the oracle."""
    l, n, s = 64, 400_000, 48
    X = np.random.default_rng(11).standard_normal((l, n))
    Js, _, Rf, st = skel.pivot_lupp(torch.from_numpy(X).to(dev), s)
    skel.check_status(st)
    ref = pivoting.lupp_columns(X, s)
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(Rf.cpu().numpy(), ref["R"])


@pytest.mark.parametrize("l,n,m,s", [(20, 100, 120, 20), (140, 3001, 2500, 130), (60, 800, 20000, 50),
                                     (70, 500, 70, 64), (8, 300, 300, 8)])
def test_pivot_skeleton_fp64_bit_exact(skel, dev, l, n, m, s):
    """Algorithm 2's column and row pivoting in one call, the row LUPP pipelined behind the
    column LUPP (row panels of a different height when C^T's panel is smaller): in FP64 the pivots and the
    column LUPP's factors equal the oracle's bit for bit."""
    rng = np.random.default_rng(l + n + m + s)
    X = rng.standard_normal((l, n))
    A = np.asfortranarray(rng.standard_normal((m, n)))
    Js, Is, Lf, Rf, st = skel.pivot_skeleton(torch.from_numpy(X).to(dev), torch.from_numpy(A).to(dev), s)
    torch.cuda.synchronize()
    skel.check_status(st)
    ref = pivoting.lupp_columns(X, s)
    assert np.array_equal(Js.cpu().numpy(), ref["Js"])
    assert np.array_equal(Rf.cpu().numpy(), ref["R"])
    assert np.array_equal(Lf.cpu().numpy(), ref["L"][:s, :s])
    assert np.array_equal(Is.cpu().numpy(), pivoting.lupp_rows(A[:, ref["Js"]], s)["Js"])


@pytest.mark.parametrize("prec", ["tf32", "f32"])
def test_pivot_skeleton_fp32_equals_separate_calls(skel, dev, prec):
    """FP32 at the measured size (8192 x 8192, k = 256, l = 272): the one-call pipelined form
    returns exactly the pivots and factors of skel_pivot_lupp followed by skel_pivot_rows."""
    m = n = 8192
    k, l = 256, 272
    A = workloads.torch_dense_spectrum(m, n, workloads.sigma_harmonic(n), 1e-6 / np.sqrt(m),
                                       workloads.seed_for("dense_8192x8192"), dev, torch.float32)
    X, st = skel.sketch(A, l, prec=prec, seed=5)
    Js1, L1, R1, _ = skel.pivot_lupp(X, k, status=st)
    Is1, _ = skel.pivot_rows(A, Js1, status=st)
    Js2, Is2, L2, R2, _ = skel.pivot_skeleton(X, A, k, status=st)
    torch.cuda.synchronize()
    skel.check_status(st)
    assert torch.equal(Js1, Js2) and torch.equal(Is1, Is2)
    assert torch.equal(L1, L2) and torch.equal(R1, R2)


def test_pivot_skeleton_rank_deficient(skel, dev):
    """A sketch with two nonzero columns and s = 30: the column LUPP stops at step 2 with
    SKEL_ERR_RANK_DEFICIENT; the row chain sees the missing pivots and leaves Is at -1 (its
    first panel needs Js[0 .. 29])."""
    X = np.zeros((40, 300))
    X[0, 7] = 2.0
    X[1, 9] = -1.0
    A = np.asfortranarray(np.random.default_rng(3).standard_normal((200, 300)))
    Js, Is, _, _, st = skel.pivot_skeleton(torch.from_numpy(X).to(dev), torch.from_numpy(A).to(dev), 30)
    torch.cuda.synchronize()
    with pytest.raises(skel.SkelError) as e:
        skel.check_status(st)
    assert e.value.code == 4
    J, I = Js.cpu().numpy(), Is.cpu().numpy()
    assert list(J[:2]) == [7, 9] and np.all(J[2:] == -1)
    assert np.all(I == -1)


def test_sketch_and_lupp_capture_into_a_cuda_graph(skel, dev):
    """The sketch and the look-ahead LUPP (two library streams forked from and joined back into
    the caller's) capture into a CUDA graph; replays give the eager call's pivots and factors."""
    m, n, l, k = 4096, 8192, 272, 256
    A = torch.randn(n, m, device=dev, generator=torch.Generator(device=dev).manual_seed(3)).t()
    X = torch.empty(l, n, device=dev)
    st = skel.new_status(dev)

    def step():
        skel.sketch(A, l, prec="tf32", seed=3, X=X, status=st)
        return skel.pivot_lupp(X, k, factors=True, status=st)

    J0, _, R0, _ = step()
    J0, R0 = J0.clone(), R0.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        step()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            out = step()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    skel.check_status(st)
    assert torch.equal(out[0], J0)
    assert torch.equal(out[2], R0)
