"""Seeded synthetic inputs shaped like the paper's experiments (Sec. 5.3) and the benchmark
configurations.  Shared by the oracle-side tests and the CUDA-side tests and bench; it holds
none of the skeletonization arithmetic (no sketch, no pivoting, no ID/CUR): only matrix
construction.

Every dense input is built in FP64 and rounded once to its storage type; the same rounded
matrix is handed to both the oracle and the GPU.

Recipes
-------
dense_spectrum     A = U diag(sigma) V^T + noise, U, V Haar (QR of a seeded Gaussian with
                   the signs fixed so that diag(R) > 0).
snn_csc            sparse non-negative A = sum_i s_i x_i y_i^T (Eq. (SNN)) with sparse
                   Uniform(0,1) factors, plus small noise on the support only.
kahan_type         X = [R_1, R_2] with R_1 unit upper triangular, -1 above the diagonal,
                   R_2 all ones: the tight case of Lemma 2.
separated_columns  A = B D with geometric column scales in random order, so that greedy
                   pivots are separated by wide relative gaps.
kernel_blocks      uneven Gaussian-kernel blocks exp(-|x - y|^2 / h^2) between
                   well-separated 3-D point clusters.
kernel_points      the same blocks' point sets (FP32), for blocks given implicitly.
"""

from .gen import *  # noqa: F401,F403
