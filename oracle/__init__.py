"""Plain FP64 CPU oracle for randomized-pivoting skeletonization (Dong & Martinsson,
"Simpler is better: a comparative study of randomized pivoting algorithms for CUR and
interpolative decompositions", arXiv 2104.05877).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  It shares no code with the CUDA
library (``paper_2104_05877_gb300``): it has its own counter-based generator, its own
Gaussian and sparse-sign transforms, textbook LU with partial pivoting, textbook column
pivoted QR, least-squares interpolation matrices and the a-posteriori error factor of
Theorem 1.  Every routine follows the paper's definitions step by step, in FP64, with no
blocking or fusion; library primitives (matmul, LAPACK QR, triangular solves, SVD) serve
only as single steps.

Modules
-------
philox      Philox-4x32-10 / 4x64-10 counter-based generator (Salmon et al., SC'11).
embedding   Gaussian embedding (Sec. 2.3, item 1) and sparse sign embedding (Sec. 2.3,
            item 3); operand-rounding emulation (FP32, BF16).
sketch      Row sketch X = Gamma A (the sketch step of Algorithms 1 and 2).
pivoting    Column-wise LUPP (Sec. 2.5.2, Eq. (LUPP)) and CPQR (Sec. 2.5.1).
decomp      Column ID  C C^+ A  (Eq. (2.1)) and stable CUR  Q_C (Q_C^T A Q_R) Q_R^T
            (Remark 3).
errors      Relative ID / CUR errors, Theorem 1's factor eta, rank-k optimum.
rank        Tolerance-driven rank for the batched blocks (a reading; the paper is silent).
skeleton    Algorithm 2 end to end (sketch -> LUPP on X -> LUPP on C -> ID/CUR).

Parity status: every function listed above is pinned by tests under ``tests/`` that check
it against facts the paper or the mathematics fixes (see each test's docstring).
"""

from . import philox, embedding, sketch, pivoting, decomp, errors, rank, skeleton  # noqa: F401
