import numpy as np
import scipy.sparse as sp

__all__ = [
    "SEED_BASE", "WORKLOAD_SEED_OFFSETS", "seed_for", "haar_orthogonal", "dense_spectrum",
    "sigma_geometric40", "sigma_harmonic", "sigma_exp200", "dense_geometric40", "dense_harmonic", "snn_csc",
    "kahan_type", "separated_columns", "exact_rank", "kernel_blocks",
    "torch_dense_spectrum", "torch_dense_exp200", "EXP200_R_EFF",
    "torch_kernel_blocks", "kernel_points"]

SEED_BASE = 2104_05877
# Seed offsets of the named workloads: seed_A = SEED_BASE + offset, seed_Gamma = seed_A + 1000.
WORKLOAD_SEED_OFFSETS = {"dense_1000x800": 1, "dense_8192x8192": 2, "snn_262144x4096": 3,
                         "kernel_blocks_4096": 4, "dense_65536x32768": 5}


def seed_for(workload, what="A"):
    """Seed of a named workload's A (what = "A") or of its embedding (what = "gamma")."""
    base = SEED_BASE + WORKLOAD_SEED_OFFSETS[workload]
    return base if what == "A" else base + 1000


def haar_orthogonal(rows, cols, rng):
    """rows x cols matrix with orthonormal columns, Haar distributed."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G, mode="reduced")
    return Q * np.sign(np.diag(R))[None, :]


def dense_spectrum(m, n, sigma, noise_std, seed, dtype=np.float64):
    """A = U diag(sigma) V^T + noise_std * N(0,1) i.i.d., built in FP64, rounded once."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = haar_orthogonal(m, r, rng)
    V = haar_orthogonal(n, r, rng)
    A = (U * np.asarray(sigma, dtype=np.float64)[None, :]) @ V.T
    if noise_std:
        A = A + noise_std * rng.standard_normal((m, n))
    return np.asfortranarray(A.astype(dtype))


def sigma_geometric40(n):
    """sigma_j = 10^(-(j-1)/40), j = 1..n."""
    return 10.0 ** (-np.arange(n) / 40.0)


def sigma_harmonic(n):
    """sigma_j = 1/j, j = 1..n."""
    return 1.0 / np.arange(1, n + 1)


def sigma_exp200(r):
    """sigma_j = exp(-j/200), j = 1..r."""
    return np.exp(-np.arange(1, r + 1) / 200.0)


def dense_geometric40(m=1000, n=800, seed=None):
    """Plain small case: 1000 x 800 FP64, sigma_j = 10^(-(j-1)/40), + 1e-12 N(0,1)."""
    seed = seed_for("dense_1000x800") if seed is None else seed
    return dense_spectrum(m, n, sigma_geometric40(min(m, n)), 1e-12, seed, np.float64)


def dense_harmonic(m, n, seed=None, floor=1e-6, dtype=np.float32):
    """sigma_j = 1/j plus a noise floor: floor * G / sqrt(m) (singular values ~ floor)."""
    seed = seed_for("dense_8192x8192") if seed is None else seed
    return dense_spectrum(m, n, sigma_harmonic(min(m, n)), floor / np.sqrt(m), seed, dtype)


def exact_rank(m, n, r, seed, dtype=np.float64, decay=0.8):
    """Exactly rank-r matrix with geometric singular values decay^j."""
    return dense_spectrum(m, n, decay ** np.arange(r), 0.0, seed, dtype)


def separated_columns(m, n, seed, ratio=0.7, dtype=np.float64):
    """A = B D: B Gaussian, D = diag(ratio^pi(j)) for a random permutation pi, so column
    magnitudes differ by at least the factor ratio between ranks."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, n))
    scales = ratio ** rng.permutation(n).astype(np.float64)
    return np.asfortranarray((B * scales[None, :]).astype(dtype))


def kahan_type(l, n):
    """X = [R_1, R_2]: R_1 (l x l) unit upper triangular with -1 above the diagonal,
    R_2 (l x (n - l)) all ones -- the tight case of Lemma 2."""
    R1 = np.eye(l) - np.triu(np.ones((l, l)), 1)
    R2 = np.ones((l, n - l))
    return np.hstack([R1, R2])


def snn_csc(m, n, r, seed, density=None, noise=1e-4, dtype=np.float32):
    """Sparse non-negative A = sum_{i<=r} s_i x_i y_i^T (Eq. (SNN)), s_i = 2/i for i <= 100
    and 1/i after (Sec. 5.3, SNN matrices).  x_i, y_i have Uniform(0,1) values on a random
    support of density d each (default d = sqrt(0.01 / r), so A is about 1% dense);
    noise * Uniform(0,1) is added on the support of A only.  Returns scipy CSC (dtype)."""
    rng = np.random.default_rng(seed)
    d = np.sqrt(0.01 / r) if density is None else density
    s = np.where(np.arange(1, r + 1) <= 100, 2.0, 1.0) / np.arange(1, r + 1)
    rows, cols, vals = [], [], []
    for i in range(r):
        xi = np.flatnonzero(rng.random(m) < d)
        yi = np.flatnonzero(rng.random(n) < d)
        if xi.size == 0 or yi.size == 0:
            continue
        xv = rng.random(xi.size)
        yv = rng.random(yi.size)
        rows.append(np.repeat(xi, yi.size))
        cols.append(np.tile(yi, xi.size))
        vals.append(s[i] * np.outer(xv, yv).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m, n)).tocsc()
    A.sum_duplicates()
    A.data = A.data + noise * rng.random(A.data.size)
    A.sort_indices()
    return A.astype(dtype)


def kernel_blocks(nblocks, seed, mrange=(64, 1024), nrange=(64, 512), h=0.5, sep=4.0,
                  dtype=np.float32):
    """Uneven Gaussian-kernel blocks exp(-|x - y|^2 / h^2) between seeded 3-D clusters of
    points (uniform in a unit cube) whose centres are `sep` apart along a random direction.
    Returns a list of Fortran-ordered arrays."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nblocks):
        mb = int(rng.integers(mrange[0], mrange[1] + 1))
        nb = int(rng.integers(nrange[0], nrange[1] + 1))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        x = rng.random((mb, 3))
        y = rng.random((nb, 3)) + sep * d
        D2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
        out.append(np.asfortranarray(np.exp(-D2 / (h * h)).astype(dtype)))
    return out


def kernel_points(nblocks, seed, mrange=(64, 1024), nrange=(64, 512), sep=4.0):
    """The point sets of kernel_blocks (same seeded draws, same order), rounded to FP32: a list
    of (x (m_b x 3), y (n_b x 3)) float32 arrays, for blocks given implicitly by their points."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nblocks):
        mb = int(rng.integers(mrange[0], mrange[1] + 1))
        nb = int(rng.integers(nrange[0], nrange[1] + 1))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        x = rng.random((mb, 3))
        y = rng.random((nb, 3)) + sep * d
        out.append((x.astype(np.float32), y.astype(np.float32)))
    return out


def torch_dense_spectrum(m, n, sigma, noise_std, seed, device, dtype):
    """Same recipe as dense_spectrum, built with torch on `device` (for full-size inputs).
    The Haar factors come from torch's QR in FP64; the result is rounded once to dtype and
    returned column-major (as the transpose view of a row-major n x m tensor)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    r = len(sigma)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)

    def haar(rows):
        G = torch.randn(rows, r, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(G, mode="reduced")
        return Q * torch.sign(torch.diagonal(R))[None, :]

    U = haar(m)
    V = haar(n)
    At = V @ (U * sig[None, :]).T            # n x m row-major == A column-major
    del U, V
    if noise_std:
        At += noise_std * torch.randn(n, m, generator=g, device=device, dtype=torch.float64)
    return At.to(dtype).t()                  # m x n view, column-major storage


EXP200_R_EFF = 3300        # exp(-3300/200) < 1e-7: below this the spectrum is the noise floor


def torch_dense_exp200(device, m=65536, n=32768, r_eff=EXP200_R_EFF, floor=1e-7, seed=None):
    """Large low-precision case: A = U diag(sigma) V^T + floor * G / sqrt(m), sigma_j =
    exp(-j/200) for j <= r_eff, U (m x r_eff) and V (n x r_eff) Haar by QR of FP32 Gaussians,
    built in FP32 on `device` (an FP64 build at 65536 x 32768 would cost ~14 FP64 TFLOP).
    Returned column-major (the transpose view of a row-major n x m tensor)."""
    import torch
    seed = seed_for("dense_65536x32768") if seed is None else seed
    sig = sigma_exp200(r_eff)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        with torch.no_grad():
            U, _ = torch.linalg.qr(torch.randn(m, r_eff, generator=g, device=device))
            V, _ = torch.linalg.qr(torch.randn(n, r_eff, generator=g, device=device))
            At = V @ (U * torch.as_tensor(sig, device=device, dtype=torch.float32)[None, :]).T   # n x m
            del U, V
            At += (floor / np.sqrt(m)) * torch.randn(n, m, generator=g, device=device)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    return At.t()


def torch_kernel_blocks(nblocks, seed, device, mrange=(64, 1024), nrange=(64, 512), h=0.5, sep=4.0):
    """Same recipe as kernel_blocks, built with torch on `device` (for the full-size batch).
    Sizes and cluster directions come from the host generator; each block is FP32, column-major,
    with a leading dimension rounded up to a multiple of 4 (16-byte aligned columns)."""
    import torch
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = []
    for _ in range(nblocks):
        mb = int(rng.integers(mrange[0], mrange[1] + 1))
        nb = int(rng.integers(nrange[0], nrange[1] + 1))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        x = torch.rand(mb, 3, generator=g, device=device, dtype=torch.float64)
        y = torch.rand(nb, 3, generator=g, device=device, dtype=torch.float64) + torch.as_tensor(sep * d, device=device)
        ld = (mb + 3) // 4 * 4
        At = torch.zeros(nb, ld, dtype=torch.float32, device=device)
        At[:, :mb] = torch.exp(-torch.cdist(y, x) ** 2 / (h * h)).to(torch.float32)
        out.append(At.t()[:mb])
    return out
