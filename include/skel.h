/*
 * skel.h -- C ABI of libskel, a GB300 (sm_103a) library for randomized-pivoting
 * skeletonization: column interpolative decomposition (ID) and CUR decomposition by
 * pivoting on a random sketch (Dong & Martinsson, "Simpler is better: a comparative study of
 * randomized pivoting algorithms for CUR and interpolative decompositions", arXiv 2104.05877).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every matrix pointer is a DEVICE pointer owned by the caller (the A of skel_sketch_host and
 *    skel_sketch_host_two_sided is a host pointer); the library never frees or retains it.
 *    Only the two batch plan constructors allocate device memory (the plan's own, freed by
 *    skel_batch_plan_destroy); every other call that needs scratch memory takes a
 *    caller-provided device workspace `ws` of `*ws_bytes` bytes (skel_pivot_lupp_static uses a
 *    fixed array inside the library instead).  Calling with ws == NULL writes the required
 *    size to *ws_bytes and returns SKEL_OK without launching anything.  A workspace smaller
 *    than required returns SKEL_ERR_WORKSPACE.  Workspace must be 256-byte aligned.
 *  - Tall matrices (A, C, Q: m rows) are COLUMN-MAJOR: element (i, j) at p[i + j*ld], ld >= m.
 *    Wide matrices (the sketch X, pivot factors R, the ID matrix Z: l or s rows, n columns)
 *    are ROW-MAJOR: element (r, j) at p[r*ld + j], ld >= n.  (So X^T is column-major n x l.)
 *  - Indices are 0-based int32 (the paper's MATLAB indices are 1-based), in selection order.
 *  - All work is enqueued on `stream` in stream order; no call synchronizes the host (except
 *    the host-A sketches with a pageable A, whose copies the driver stages through the host).
 *    Argument errors are detected on the host and returned synchronously with nothing
 *    launched.  Errors found on the device (non-finite data, a zero pivot, a timed-out grid
 *    wait) are written to `dev_status` (device int32[2]: {code, step}; may be NULL), first
 *    error wins; the caller reads it after synchronizing.  Device errors never trap.
 *  - Random numbers: every entry of an embedding is a function of (seed, row, column) through
 *    Philox-4x32-10 (Salmon et al., SC'11), so the same seed gives the same embedding in any
 *    launch shape.
 *  - Library-owned streams and events (the look-ahead streams of skel_pivot_lupp, the
 *    auxiliary stream of skel_pivot_skeleton and skel_id_cur, the copy stream of the host-A
 *    sketches) are created by the first call that needs them in each CUDA context and device,
 *    and kept under that context's unique id (cuCtxGetId).  After cudaDeviceReset, or from
 *    another context, the next call creates new ones; those of a destroyed context are not
 *    released.  Make the first such call before any stream capture.
 */
#ifndef SKEL_H
#define SKEL_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SKEL_OK = 0,
  SKEL_ERR_INVALID_ARG = 1,    /* host-side argument check failed; nothing launched        */
  SKEL_ERR_WORKSPACE = 2,      /* *ws_bytes smaller than required, or ws misaligned        */
  SKEL_ERR_NONFINITE = 3,      /* device: NaN/Inf met in the data                          */
  SKEL_ERR_RANK_DEFICIENT = 4, /* device: an exactly zero pivot; dev_status[1] = its step  */
  SKEL_ERR_TIMEOUT = 5,        /* device: a grid-wide wait exceeded its limit              */
  SKEL_ERR_CUDA = 6,           /* a CUDA runtime call failed (launch, attribute, memset)   */
  SKEL_ERR_UNSUPPORTED = 7     /* valid request the library does not implement              */
} skel_status;

/* storage type of a matrix */
typedef enum { SKEL_F64 = 0, SKEL_F32 = 1 } skel_dtype;

/* arithmetic of the sketch product: operands rounded to this format, products accumulated
 * in FP32 (FP64 for SKEL_PREC_F64). */
typedef enum {
  SKEL_PREC_F64 = 0,  /* plain: FP64 operands and accumulation (SIMT DFMA)                */
  SKEL_PREC_F32 = 1,  /* FP32 operands and accumulation (SIMT FFMA)                       */
  SKEL_PREC_TF32 = 2, /* tensor cores (tcgen05 kind::tf32), FP32 accumulate in TMEM       */
  SKEL_PREC_BF16 = 3, /* tensor cores (tcgen05 kind::f16, bf16 operands), FP32 accumulate */
  SKEL_PREC_FP8 = 4   /* tensor cores (tcgen05 kind::f8f6f4, e4m3 operands; A with one
                         power-of-two scale per column), FP32 accumulate                        */
} skel_prec;

/* embedding Gamma (Sec. 2.3) */
typedef enum {
  SKEL_SKETCH_GAUSSIAN = 0,    /* i.i.d. N(0, 1/l) (Sec. 2.3, item 1)                        */
  SKEL_SKETCH_SPARSE_SIGN = 1, /* zeta +-1/sqrt(zeta) per column at distinct rows (item 3)   */
  SKEL_SKETCH_SRTT = 2         /* sqrt(m/l) Pi_{m->l} T Phi Pi_{m->m}, T the unitary discrete
                                  Hartley transform (item 2)                                  */
} skel_sketch_kind;

const char* skel_status_string(int status);
int skel_version(void);
/* Number of CUDA kernels this library has launched in the calling process so far. */
uint64_t skel_launch_count(void);

/*
 * skel_sketch -- row sketch X = Gamma A of a dense A (the sketch step of Algorithms 1 and 2;
 * Table 1).
 *   m, n      : A is m x n, column-major, leading dimension lda >= m, storage a_dtype.
 *   l         : number of sketch rows (l = k + p, Sec. 2.3), 1 <= l <= 4096.
 *   kind      : Gaussian (Gamma(i,j) = G(i,j)/sqrt(l), G from Philox + Box-Muller with
 *               counter (j/4, i, 0, 0)) or sparse sign (zeta nonzeros per column, Floyd's
 *               sampling from counters (j, 0, 1, c)) or SRTT; zeta is ignored for Gaussian
 *               and SRTT.  SRTT: Gamma(i, q) = phi_r cas(2 pi sel(i) r / m) / sqrt(l) with
 *               r = pi^{-1}(q); pi and sel are keyed Feistel permutations of 0..m-1 (4 rounds
 *               on 2h bits, 4^h >= m, round function Philox word x of counter (R, round, tag,
 *               0) masked to h bits, tags 2 and 3, cycle walking onto 0..m-1), sel(i) for
 *               i < l, and phi_r = -1 when bit 0 of Philox word x of counter (r, 0, 4, 0) is
 *               set.  SRTT needs 1 <= l <= m < 2^31 (SKEL_ERR_INVALID_ARG otherwise),
 *               supports F64, F32, TF32 and BF16, and no row offset (skel_sketch_rows with
 *               row0 > 0 returns SKEL_ERR_UNSUPPORTED).
 *   prec      : arithmetic of the product (skel_prec).  SKEL_PREC_F64 requires
 *               a_dtype = SKEL_F64 and writes X as FP64; every other precision reads A as
 *               stored and writes X as FP32.  Sparse sign supports F64 and F32 only.  The
 *               tensor-core precisions (TF32, BF16, FP8) need a_dtype = SKEL_F32, a 16-byte
 *               aligned A and lda a multiple of 4 (A is streamed by TMA); otherwise they
 *               return SKEL_ERR_UNSUPPORTED.
 *   X, ldx    : output, l x n row-major (ldx >= n).
 * The Gaussian entries (and the SRTT's, on the tensor-core path) are generated inside the
 * kernel and never stored; the SRTT's F64 / F32 path stores the l x m Gamma in the
 * workspace.  Non-finite
 * entries of X set SKEL_ERR_NONFINITE in dev_status.
 */
skel_status skel_sketch(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda,
                        int32_t l, skel_sketch_kind kind, int32_t zeta, skel_prec prec,
                        uint64_t seed, void* X, int64_t ldx, void* ws, size_t* ws_bytes,
                        int32_t* dev_status, cudaStream_t stream);

/*
 * skel_sketch_rows -- the partial sketch of a block of rows of a larger A (the row-partitioned
 * form of Algorithm 2's sketch step: X = sum over row blocks of Gamma(:, rows) A(rows, :)).
 *   row0      : global index of the block's first row; a multiple of 4, row0 + m <= 2^32 - 1.
 *               Gamma's columns row0 .. row0+m-1 are generated (Gaussian counters (j/4, i, 0, 0)
 *               and sparse-sign counters (j, 0, 1, c) use the global row j), so the partial
 *               sketches of a partition of A's rows sum to skel_sketch of the whole A.
 *   every other argument is skel_sketch's, for the m x n block (A points at its first row).
 * skel_sketch(...) is skel_sketch_rows(0, ...).  Errors: SKEL_ERR_INVALID_ARG for a negative
 * or unaligned row0, else as skel_sketch.
 */
skel_status skel_sketch_rows(int64_t row0, int64_t m, int64_t n, skel_dtype a_dtype, const void* A,
                             int64_t lda, int32_t l, skel_sketch_kind kind, int32_t zeta, skel_prec prec,
                             uint64_t seed, void* X, int64_t ldx, void* ws, size_t* ws_bytes,
                             int32_t* dev_status, cudaStream_t stream);

/*
 * skel_sketch_host -- skel_sketch of an A that lives in host memory, streamed to the device in
 * column panels.  X = Gamma A reads A once (Algorithm 1, sketch step; the single pass over A of
 * Sec. 2.3), and X's columns j0..j1 depend on A's columns j0..j1 only, so the copy of one panel
 * overlaps the sketch of the one before: panels go through two device staging buffers in the
 * workspace, copied on a library-owned stream and sketched on `stream`.  A never has to fit
 * in device memory.
 *   A, lda    : m x n column-major in host memory (a device pointer also works).  Page-locked
 *               (pinned) memory gives asynchronous copies that overlap the sketch; pageable
 *               memory is accepted, and the driver then stages each panel copy through the
 *               host, which may block the calling thread.
 *   panel     : columns per panel; 0 chooses about 512 MiB of A per panel (a multiple of 256
 *               columns, of 4 when columns are taller than 2 MiB, at least one column).
 *   every other argument is skel_sketch's; the tensor-core precisions need no alignment of the
 *               host A (the staging columns are padded to 16 bytes).
 * X equals skel_sketch of the same A on the device up to the summation order of the K-split
 * partial sums, which depends on the panel width.  Workspace: two staging panels of
 * esize * round_up(m, 4) * panel bytes plus skel_sketch's workspace for one panel.  The call
 * enqueues its work and returns (pinned A); the caller must keep A unchanged until `stream`
 * reaches the end of the call's work.  Errors: as skel_sketch; SKEL_ERR_INVALID_ARG for a
 * negative panel.
 */
skel_status skel_sketch_host(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                             skel_sketch_kind kind, int32_t zeta, skel_prec prec, uint64_t seed, void* X,
                             int64_t ldx, int64_t panel, void* ws, size_t* ws_bytes, int32_t* dev_status,
                             cudaStream_t stream);

/*
 * skel_sketch_host_two_sided -- both sketches of the streaming skeleton selection (Algorithm 3)
 * from ONE pass over an A in host memory: X = Gamma A (l x n, as skel_sketch with the
 * Gaussian embedding and seed_gamma) and Yt = Omega A^T (l x m, as skel_sketch_cols with
 * seed_omega).  Each column panel A(:, j0:j0+w) is copied to the device once (as in
 * skel_sketch_host) and gives X(:, j0:j0+w) = Gamma A(:, panel) and the partial sum
 * Omega(:, j0:j0+w) A(:, panel)^T of Yt, which the library adds up across panels (the first
 * panel writes Yt, later ones add a partial).  This is the single-pass form Algorithm 3 is
 * designed for: A is seen once, and neither A nor a transposed copy of it is kept on the device.
 *   m, n >= 1; l in 1..4096; prec: SKEL_PREC_F64 (a_dtype F64), SKEL_PREC_F32, SKEL_PREC_TF32 or
 *               SKEL_PREC_BF16 (a_dtype F32).  The tensor-core precisions transpose each panel on
 *               the device and run the tensor-core sketch with Omega's column offset j0.
 *   panel     : columns per panel, a multiple of 4 (Omega's counters take columns four at a
 *               time); 0 chooses about 512 MiB of A per panel.
 *   X, ldx    : l x n row-major (ldx >= n).   Yt, ldy: l x m row-major (ldy >= m).
 * X and Yt equal skel_sketch and skel_sketch_cols on the device copy of A up to the order of
 * their sums.  Workspace: two staging panels, the row sketch's workspace for one panel, the
 * column sketch's (plus a transposed panel for TF32 / BF16) and one l x m partial.  A must stay
 * unchanged until `stream` reaches the end of the call's work.  Errors: SKEL_ERR_INVALID_ARG for
 * bad sizes, a panel that is negative or not a multiple of 4, or a_dtype not matching prec;
 * SKEL_ERR_UNSUPPORTED for FP8; non-finite entries set SKEL_ERR_NONFINITE in dev_status.
 */
skel_status skel_sketch_host_two_sided(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda,
                                       int32_t l, skel_prec prec, uint64_t seed_gamma, uint64_t seed_omega, void* X,
                                       int64_t ldx, void* Yt, int64_t ldy, int64_t panel, void* ws, size_t* ws_bytes,
                                       int32_t* dev_status, cudaStream_t stream);

/*
 * skel_sketch_cols -- the column sketch of the streaming skeleton selection (Algorithm 3):
 *     Y = A Omega^T (m x l),  Omega l x n Gaussian with N(0, 1/l) entries,
 * returned transposed, Yt = Omega A^T (l x m row-major, ldy >= m), so that the row skeletons
 * I_s are the column pivots of skel_pivot_lupp on Yt (Algorithm 3, row pivoting).  Omega's counters
 * are those of the Gaussian embedding over n columns (column j of Omega pairs with column j of
 * A); use a seed different from Gamma's for an independent Omega.  prec: SKEL_PREC_F64
 * (a_dtype F64) or SKEL_PREC_F32 (a_dtype F32), on the SIMT path with Omega generated in the
 * kernel.  Workspace: GEMM split-K scratch (handshake).
 */
skel_status skel_sketch_cols(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                             skel_prec prec, uint64_t seed, void* Yt, int64_t ldy, void* ws, size_t* ws_bytes,
                             int32_t* dev_status, cudaStream_t stream);

/*
 * skel_sketch_power -- row space approximator with q plain power iterations (Sec. 3,
 * Eq. (def_power_iter); Rand-LUPP-1piter of Sec. 5 is q = 1):
 *     X = Omega (A^T A)^q,   Omega l x n Gaussian with N(0, 1/l) entries,
 * formed as X = (Omega A^T) A, then q - 1 times X <- (X A^T) A, without orthogonalisation
 * (the plain form the paper times; it loses accuracy for ill-conditioned A when q > 1).
 * Omega's counters are those of the Gaussian embedding with n in place of m (column j of
 * Omega pairs with column j of A).  1 <= q <= 8.
 *   prec: SKEL_PREC_F64 (a_dtype F64, FP64 throughout), SKEL_PREC_F32 or SKEL_PREC_TF32
 *   (a_dtype F32; Omega A^T on the FP32 SIMT path, (.) A on the tensor cores with FP32
 *   accuracy (3xTF32) when A is TMA-addressable, else FP32 SIMT).  X: l x n row-major.
 * Two passes over A per iteration; workspace l m words plus GEMM scratch (handshake).
 */
skel_status skel_sketch_power(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                              int32_t q, skel_prec prec, uint64_t seed, void* X, int64_t ldx, void* ws,
                              size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_sketch_csc -- X = Gamma A for a sparse A in compressed sparse column form (Table 1,
 * T_s = O(nnz(A) zeta) for the sparse sign embedding).
 *   col_ptr[n+1] (int64), row_idx[nnz] (int32, any order within a column), val[nnz] (FP32).
 *   kind must be SKEL_SKETCH_SPARSE_SIGN or SKEL_SKETCH_GAUSSIAN.  X is FP32, l x n
 *   row-major.
 */
skel_status skel_sketch_csc(int64_t m, int64_t n, int64_t nnz, const int64_t* col_ptr,
                            const int32_t* row_idx, const float* val, int32_t l,
                            skel_sketch_kind kind, int32_t zeta, uint64_t seed, float* X,
                            int64_t ldx, void* ws, size_t* ws_bytes, int32_t* dev_status,
                            cudaStream_t stream);

/*
 * skel_pivot_lupp -- column-wise LU with partial pivoting on X (Sec. 2.5.2, Eq. (LUPP);
 * Algorithm 2, column pivoting), first s steps.  Step t picks j_t = argmax over unselected j of
 * |S(t, j)| for the current Schur complement S (ties: lowest column index), then
 * R(t, :) = S(t, :)/S(t, j_t) and S(t+1:, :) -= S(t+1:, j_t) R(t, :).  Only rows 0..s-1 of X
 * are read.  Row pivoting of a tall C (Algorithm 2) is this call on C^T: pass the
 * column-major m x s C as X with l = s, n = m, ldx = ldc.
 *   dtype     : storage and arithmetic of X and of the factors (F64 or F32).
 *   X, ldx    : l x n row-major input (not modified).  1 <= s <= min(l, n), s <= 1024.
 *   Js        : out, int32[s], pivots in selection order.
 *   L, ldl    : optional out (may be NULL), s x s lower triangular, row-major, L(r, t) =
 *               S(r, j_t) at step t; X(0:s, :) = L R.
 *   R, ldr    : optional out (may be NULL), s x n row-major, R(t, j_t) = 1, |R| <= 1.
 * A zero pivot at step t sets SKEL_ERR_RANK_DEFICIENT with step t and writes Js[t..] = -1.
 */
skel_status skel_pivot_lupp(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx,
                            int32_t s, int32_t* Js, void* L, int64_t ldl, void* R, int64_t ldr,
                            void* ws, size_t* ws_bytes, int32_t* dev_status,
                            cudaStream_t stream);

/*
 * skel_pivot_lupp_static -- the LUPP of skel_pivot_lupp (same arguments, same outputs) for
 * callers that cannot allocate device memory.  Some programs must not allocate: a host that
 * hands out all device memory from its own fixed pool and forbids allocations after start-up,
 * or a loop with a hard latency budget where cudaMalloc's implicit synchronisation of the
 * whole device is not acceptable.  Such a caller passes only X and the outputs; this entry
 * point allocates nothing.  (The paper has no counterpart; this is an interface choice of
 * this library.)
 *   Kernel: always the persistent grid-barrier LUPP kernel (skel_pivot_lupp picks the
 *   cluster panel kernel when a panel fits a thread-block cluster).  Both kernels apply, to
 *   every entry, the operations of the LUPP step in the textbook order with the same
 *   arithmetic (FP64: separately rounded divide, multiply and subtract; FP32: a fused
 *   multiply-subtract per update and a multiply by the correctly rounded reciprocal of the
 *   pivot), so Js, L and R are bitwise equal to skel_pivot_lupp's; the two differ in speed
 *   only.
 *   Scratch: a fixed 8 MiB array in the library's device image, held by every device that
 *   loads the library until the process exits.  A problem whose scratch need exceeds 8 MiB
 *   (e.g. FP64 with l = s = n = 996; 992 still fits) returns SKEL_ERR_WORKSPACE with nothing
 *   launched.
 *   Set-up: the first call in a CUDA context, with that context current, looks up the array's
 *   device address (cudaGetSymbolAddress) and caches it under the context's unique id; make
 *   that first call before any stream capture.  Later calls in the same context do no set-up.
 *   After cudaDeviceReset (the array may move when the library's module is loaded again) or
 *   from another context, the next call finds no cached address and looks it up again.
 *   Sharing: every call on a device uses the same array and each call leaves its contents
 *   behind; a call clears what must start at zero itself.  Calls that overlap on the GPU
 *   (different streams, or host threads, without ordering between them) race on the array
 *   and give wrong results: order them.
 */
skel_status skel_pivot_lupp_static(skel_dtype dtype, const void* X, int64_t l, int64_t n,
                                   int64_t ldx, int32_t s, int32_t* Js, void* L, int64_t ldl,
                                   void* R, int64_t ldr, int32_t* dev_status,
                                   cudaStream_t stream);

/*
 * skel_pivot_cpqr -- column pivoted Householder QR on X (Sec. 2.5.1, Eq. (QRCP)), first s
 * steps: j_t = argmax of the remaining column norm over rows t..l-1 (kept by downdating,
 * recomputed when cancellation exceeds sqrt(unit roundoff)), then a Householder reflector
 * with beta = -sign(S(t, j_t)) ||S(t:, j_t)||.
 *   X, ldx    : l x n row-major (all l rows are read).  1 <= s <= min(l, n), l <= 1024.
 *   Js        : out int32[s].   R, ldr: optional s x n row-major, R(t, j_t) = beta_t.
 */
skel_status skel_pivot_cpqr(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx,
                            int32_t s, int32_t* Js, void* R, int64_t ldr, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_id -- column ID A ~ C Z with C = A(:, Js) (Eq. (2.1)): Z = C^+ A = R_C^{-1} Q_C^T A,
 * where C = Q_C R_C is a Householder QR (FP64 for dtype F64; FP32 for F32) and the s x s
 * triangular solve is FP64.  Z(:, Js) = I.
 *   A, lda    : m x n column-major, dtype F64 or F32.  Js: int32[s] device, distinct.
 *   Z, ldz    : out, s x n row-major FP64 (ldz >= n).
 *   sq_norms  : optional out (may be NULL), device double[2] = {||A||_F^2, ||Q_C^T A||_F^2};
 *               their difference is ||A - C Z||_F^2 (orthogonal projection).
 */
skel_status skel_id(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                    int32_t s, const int32_t* Js, double* Z, int64_t ldz, double* sq_norms,
                    void* ws, size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_id_refine -- the column ID of skel_id for an FP32 A, followed by one step of iterative
 * refinement in FP64 (corrected seminormal equations): with C = Q_C R_C the FP32 Householder
 * QR of skel_id and Z0 = R_C^{-1} Q_C^T A,
 *     Z1 = Z0 + R_C^{-1} R_C^{-T} (C^T A - (C^T C) Z0),
 * where C^T A and C^T C are formed from exact FP32 x FP32 products summed in float-float pairs
 * (about 44 significant bits, on the FP32 pipes), and the product with Z0 and both triangular
 * solves are FP64.  The step contracts the error of Z0 (about cond(C) u_32 relative) by about
 * cond(C)^2 u_32, leaving Z1 within a small multiple of cond(C)^2 u_64 of C^+ A in practice.
 * Eq. (2.1); the refinement is this library's mixed-precision design, not the paper's.
 *   Arguments, outputs and workspace handshake as skel_id (Z: s x n row-major FP64, Z(:, Js) = I;
 *   sq_norms from the unrefined W).  dtype must be SKEL_F32 (SKEL_ERR_UNSUPPORTED otherwise: an
 *   FP64 skel_id has nothing to refine at this precision).
 */
skel_status skel_id_refine(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                           int32_t s, const int32_t* Js, double* Z, int64_t ldz, double* sq_norms,
                           void* ws, size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_pivot_rows -- row skeletons of Algorithm 2 (row pivoting): gathers C = A(:, Js) (m x s) and
 * runs row-wise LUPP on it (the LUPP of skel_pivot_lupp applied to C^T).
 *   Is        : out int32[s] row skeletons in selection order.
 */
skel_status skel_pivot_rows(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                            int32_t s, const int32_t* Js, int32_t* Is, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_pivot_skeleton -- both skeletons of Algorithm 2 (column and row pivoting) in one call: the
 * column LUPP of skel_pivot_lupp on X (Js, optional L and R), then the row LUPP of
 * skel_pivot_rows on C = A(:, Js) (Is), with results identical to those two calls.  The row
 * LUPP runs behind the column LUPP panel by panel: its panel of steps [t0, t0+b) needs only
 * Js[0 .. t0+b), so it is factored on an auxiliary stream as soon as the column panel that
 * ends those pivots is done; the caller's stream waits for both chains at the end.
 *   dtype     : of X and of A (the same for both).
 *   X, l, n, ldx : the sketch, l x n row-major;  A, m, lda : m x n column-major.
 *   s         : skeletons, 1 <= s <= min(l, m, n, 1024).
 *   Js, Is    : out int32[s];  L, R : optional, as skel_pivot_lupp.
 * The auxiliary stream and its events are created once per context and device and shared by
 * every call (calls are enqueued one at a time under a lock).  When a panel of either LUPP does not fit
 * a thread-block cluster the two LUPPs run one after the other on the caller's stream.  A
 * column LUPP that stops early (rank-deficient X) leaves Is at -1.
 */
skel_status skel_pivot_skeleton(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                                const void* A, int64_t m, int64_t lda, int32_t* Js, int32_t* Is, void* L,
                                int64_t ldl, void* R, int64_t ldr, void* ws, size_t* ws_bytes, int32_t* dev_status,
                                cudaStream_t stream);

/*
 * skel_cur -- CUR A ~ C U R (Eq. (2.4)) with C = A(:, Js), R = A(Is, :) and U from the
 * stable form of Remark 3: U = R_C^{-1} (Q_C^T A Q_R) R_R^{-T}, where C = Q_C R_C and
 * R^T = Q_R R_R (Householder QR, FP64 for dtype F64, FP32 for F32; FP64 solves).
 *   Is        : row skeletons; input when rows_given != 0, otherwise computed here by
 *               row-wise LUPP on C (Algorithm 2, row pivoting) and written.
 *   U, ldu    : out s x s row-major FP64.
 *   sq_norms  : optional out (may be NULL), device double[2] = {||A||_F^2, ||Q_C^T A Q_R||_F^2};
 *               their difference is ||A - C U R||_F^2 (a two-sided orthogonal projection).
 */
skel_status skel_cur(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                     int32_t s, const int32_t* Js, int32_t* Is, int rows_given, double* U,
                     int64_t ldu, double* sq_norms, void* ws, size_t* ws_bytes,
                     int32_t* dev_status, cudaStream_t stream);

/*
 * skel_cur_refine -- the stable CUR of skel_cur for an FP32 A, followed by one step of
 * iterative refinement of U in FP64 (the two-sided form of skel_id_refine's step): with
 * C = Q_C R_C and R^T = Q_R R_R the FP32 Householder QRs of skel_cur and U0 its core,
 *     U1 = U0 + (R_C^T R_C)^{-1} (C^T A R^T - (C^T C) U0 (R R^T)) (R_R^T R_R)^{-1},
 * where C^T A, C^T C and R R^T are formed from exact FP32 products summed in float-float pairs
 * and (C^T A) R^T, the s x s products and the four triangular solves are FP64.  Eq. (2.4),
 * Remark 3; the refinement is this library's mixed-precision design, not the paper's.
 *   Arguments, outputs and workspace handshake as skel_cur (sq_norms from the unrefined
 *   W Q_R).  dtype must be SKEL_F32 (SKEL_ERR_UNSUPPORTED otherwise).
 */
skel_status skel_cur_refine(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                            int32_t s, const int32_t* Js, int32_t* Is, int rows_given, double* U,
                            int64_t ldu, double* sq_norms, void* ws, size_t* ws_bytes,
                            int32_t* dev_status, cudaStream_t stream);

/*
 * skel_error -- Frobenius errors formed directly from the residuals, and Theorem 1's
 * a-posteriori factor.
 *   out[0] = ||A||_F
 *   out[1] = ||A - A(:, Js) Z||_F                (if Z != NULL, else NaN)
 *   out[2] = ||A - A(:, Js) U A(Is, :)||_F        (if U != NULL and Is != NULL, else NaN)
 *   out[3] = eta = sqrt(1 + ||R_1^{-1} R_2||_2^2) (if Rf != NULL, else NaN), R_1 = Rf(:, Js),
 *            R_2 = the other columns of the s x n pivot factor Rf (LUPP's R or CPQR's R).
 *   out       : device double[4].
 * Products use the storage precision of A (FP32 products, FP64 sums for F32 data).
 */
skel_status skel_error(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                       int32_t s, const int32_t* Js, const double* Z, int64_t ldz,
                       const int32_t* Is, const double* U, int64_t ldu, skel_dtype rf_dtype,
                       const void* Rf, int64_t ldrf, double* out, void* ws, size_t* ws_bytes,
                       int32_t* dev_status, cudaStream_t stream);

/*
 * skel_id_cur -- the column ID of skel_id and the stable CUR of skel_cur (Eq. (2.1),
 * Eq. (2.4), Remark 3) in one call, for given skeletons Js and Is (e.g. from
 * skel_pivot_skeleton).  The QR of C = A(:, Js) and W = Q_C^T A are formed once and serve
 * both (Z = R_C^{-1} W, U = R_C^{-1} (W Q_R) R_R^{-T}); the QR of R^T = A(Is, :)^T runs on the
 * auxiliary stream concurrently with them.  Outputs and their layouts are those of skel_id
 * (Z, ldz, sq_id) and skel_cur (U, ldu, sq_cur), and equal them.  sq_id / sq_cur may be NULL.
 * Workspace (handshake).  The auxiliary stream is shared as in skel_pivot_skeleton.
 */
skel_status skel_id_cur(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                        const int32_t* Js, const int32_t* Is, double* Z, int64_t ldz, double* U, int64_t ldu,
                        double* sq_id, double* sq_cur, void* ws, size_t* ws_bytes, int32_t* dev_status,
                        cudaStream_t stream);

/*
 * skel_cur_sketch -- the CUR estimated without a second pass over A (Sec. 4: with the skeletons
 * S = A(I_s, J_s), C = A(:, J_s) and R = A(I_s, :), A ~ C S^{-1} R): U = S^{-1} (s x s row-major
 * FP64, ldu >= s), formed stably from a Householder QR of S^T (S^T = Q R_S, S^{-1} = Q R_S^{-T}).
 * Reads only C's rows I_s.  Less accurate than skel_cur's U = C^+ A R^+ (the paper notes the
 * compromise); S singular gives a non-finite U.  Arguments as skel_cur; workspace (handshake).
 */
skel_status skel_cur_sketch(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                            const int32_t* Js, const int32_t* Is, double* U, int64_t ldu, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_id_sketch -- column ID coefficients from the sketch alone, without a second pass over
 * A (Sec. 4: C^+ A ~ X_1^+ X with X_1 = X(:, J_s)), the pseudo-inverse taken over all l rows of
 * the sketch:
 *     Z = X(:, J)^+ X = argmin_Z ||X(:, J) Z - X||_F = argmin_Z ||Gamma (C Z - A)||_F,
 * the sketched least-squares problem for C^+ A (with l = s it is X(:, J)^{-1} X).  Formed as
 * X(:, J) = Q R_1 (Householder QR, the dtype's precision), W = Q^T X, Z = R_1^{-1} W (FP64
 * solve), then Z(:, J) = I exactly.
 *   X, l, n, ldx : the sketch, l x n row-major (ldx >= n), dtype FP32 or FP64.
 *   s, Js        : int32[s] distinct column indices (device), s <= l, s <= min(n, 1024).
 *   Z, ldz       : out, s x n row-major FP64 (ldz >= n).
 * Workspace (handshake).  Less accurate than skel_id (the sketch's precision and the
 * embedding's distortion enter Z); A is not read.  A rank-deficient X(:, J) gives a non-finite
 * Z (SKEL_ERR_NONFINITE from the solve's checks).
 */
skel_status skel_id_sketch(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                           const int32_t* Js, double* Z, int64_t ldz, void* ws, size_t* ws_bytes,
                           int32_t* dev_status, cudaStream_t stream);

/*
 * Batched skeletonization of many independent blocks (hierarchical-matrix compression; the
 * tolerance-driven rank is a reading: the paper fixes k).  Per block A_b (m_b x n_b, FP32,
 * column-major, device): the Gaussian sketch X_b = Gamma A_b with l = kmax + p rows (one Gamma
 * for every block, Gamma(:, 0:m_b)), computed to FP32 accuracy on the tensor cores; column LUPP
 * on X_b (Sec. 2.5.2) stopped at the smallest t <= kmax with
 *     ||S_t||_F^2 l/(l - t) <= tol^2 ||X_b||_F^2     (S_t: Schur complement after t steps)
 * (or at kmax, or at a zero pivot); and the column ID coefficients from the sketch alone,
 *     Z_b = X_b(:, J)^+ X_b = argmin_Z ||X_b(:, J) Z - X_b||_F   (C^+ A ~ X_1^+ X, Sec. 4, no second
 * pass over A; the pseudo-inverse over all l rows, by an FP32 Householder QR of X_b(:, J)).
 * A is read once.
 *
 * skel_batch_plan_create -- m, n, A, lda: host arrays of nblocks block descriptors (A[b] a
 *   device pointer, 16-byte aligned, lda[b] >= m[b] and a multiple of 4); 1 <= kmax <= 128,
 *   p >= 1, kmax + p <= 256, tol >= 0; seed as for skel_sketch.  The plan keeps the pointers
 *   (the blocks must stay allocated while it is used) and owns its device memory: tensor
 *   maps, work lists, the Gamma halves (2 (kmax+p) max(m_b) floats) and the sketches
 *   (sum_b (kmax+p) n_b floats).  Allocates and copies synchronously; no other call does.
 *   SKEL_ERR_UNSUPPORTED when a block is wider than four CTAs' shared memory hold
 *   ((kmax+p) n_b / 4 floats per CTA) or is not TMA-addressable.
 *   flags: SKEL_BATCH_AUTOTUNE times, on the plan's own blocks, every sketch pipeline depth
 *   that fits and the LUPP cluster classes run one after another or concurrently (one
 *   warm-up and two timed runs each, synchronously, inside this call) and keeps the fastest;
 *   no choice changes any result.  SKEL_BATCH_GRAPH makes skel_batch_run replay a CUDA
 *   graph of the run, captured on its first call and again whenever the output pointers
 *   change.  Other bits: SKEL_ERR_INVALID_ARG.
 * skel_batch_plan_create_points -- the same batch for blocks given implicitly (Sec. 1: the
 *   method needs A only through the entries it evaluates and the products it forms; the
 *   experiments on SNN1e6 in Sec. 5 access A only through products): block b is the
 *   Gaussian-kernel matrix A_b(i, j) = exp(-||x_i - y_j||^2 / h^2) between point sets
 *   x[b] (m[b] x dim) and y[b] (n[b] x dim), device pointers, row-major FP32 (point i's
 *   coordinates at x[b][i*dim .. i*dim + dim)), 1 <= dim <= 3, h > 0.  A_b is never stored:
 *   the sketch kernel evaluates its entries tile by tile in shared memory from per-point
 *   records the run forms first ({coordinates, -||p||^2/h^2 as a pair of floats}, 32 bytes
 *   per point, owned by the plan), the exponent -||x - y||^2/h^2 = c_x + c_y + (2/h^2) x.y
 *   as a pair of floats and the entry as expf of its leading part times (1 + its trailing
 *   part), so every entry is within a few FP32 roundings of the exact kernel value.  Z and
 *   the pivots come from the sketch alone, so no A_b exists anywhere.  The points are read
 *   at every run (they must stay allocated and may change between runs); all other
 *   arguments, errors and outputs are those of skel_batch_plan_create / skel_batch_run.
 * skel_batch_copy_sketch -- enqueues on `stream` a device-to-device copy of block b's sketch
 *   X_b ((kmax+p) x n_b, row-major FP32, as the last run left it) into X (device, caller's).
 *   For tests and diagnostics.
 * skel_batch_plan_info -- host: info[0] sketch pipeline depth, info[1] 1 if the LUPP classes
 *   run concurrently, info[2] the flags, info[3] sketch work items (128-column tiles).
 * skel_batch_z_offsets -- host: offsets[0..nblocks] (in doubles) of the blocks' Z in Z_all,
 *   offsets[b+1] - offsets[b] = kmax n_b.
 * skel_batch_run -- on `stream`, no host synchronisation: Js[b*kmax + q] (int32, q < rank_b,
 *   -1 after), ranks[b], Z_all + offsets[b]: kmax x n_b row-major FP64, rows 0 .. rank_b-1
 *   written (Z_b(:, Js) = I), rows from rank_b on left as they were.  dev_status: SKEL_ERR_NONFINITE (step = block) for a non-finite sketch,
 *   SKEL_ERR_TIMEOUT if a pipeline wait of the sketch kernel gave up.  With SKEL_BATCH_GRAPH
 *   (and per-kernel timing off) the run is one graph launch; the plan's side streams and
 *   events make the graph, so one plan serves one run at a time.
 * skel_batch_plan_destroy -- frees the plan (after the work using it has finished).
 */
typedef struct skel_batch_plan skel_batch_plan;
enum { SKEL_BATCH_GRAPH = 1, SKEL_BATCH_AUTOTUNE = 2 };
skel_status skel_batch_plan_create(int32_t nblocks, const int64_t* m, const int64_t* n, const float* const* A,
                                   const int64_t* lda, int32_t kmax, int32_t p, double tol, uint64_t seed,
                                   int32_t flags, skel_batch_plan** plan);
skel_status skel_batch_plan_create_points(int32_t nblocks, const int64_t* m, const int64_t* n, int32_t dim,
                                          const float* const* x, const float* const* y, double h, int32_t kmax,
                                          int32_t p, double tol, uint64_t seed, int32_t flags,
                                          skel_batch_plan** plan);
skel_status skel_batch_copy_sketch(const skel_batch_plan* plan, int32_t b, float* X, cudaStream_t stream);
skel_status skel_batch_plan_info(const skel_batch_plan* plan, int32_t* info);
skel_status skel_batch_z_offsets(const skel_batch_plan* plan, int64_t* offsets);
skel_status skel_batch_run(skel_batch_plan* plan, int32_t* Js, int32_t* ranks, double* Z, int32_t* dev_status,
                           cudaStream_t stream);
void skel_batch_plan_destroy(skel_batch_plan* plan);

/*
 * skel_debug_gaussian -- writes the standard normals G (l x m, row-major, ld = m) that the
 * Gaussian sketch kernels generate, in FP32 (as_fp64 = 0) or FP64 (as_fp64 = 1).  For tests
 * of the generator; the sketch kernels themselves never store G.
 */
skel_status skel_debug_gaussian(int32_t l, int64_t m, uint64_t seed, int as_fp64, void* G,
                                cudaStream_t stream);

/*
 * skel_debug_philox -- raw Philox-4x32-10 words for `count` counters (uint32[count*4] in,
 * uint32[count*4] out, device), key (k0, k1).  For tests of the generator.
 */
skel_status skel_debug_philox(const uint32_t* counters, int64_t count, uint32_t k0, uint32_t k1,
                              uint32_t* out, cudaStream_t stream);

/*
 * skel_debug_curand_philox -- cuRAND's own device Philox4_32_10 stream (curand_init(seed,
 * subsequence = i, offset 0), then per_seq calls of curand4) for i < nseq, written as
 * uint32[nseq * per_seq * 4].  Lets tests compare this library's generator with cuRAND's.
 */
skel_status skel_debug_curand_philox(uint64_t seed, int64_t nseq, int per_seq, uint32_t* out,
                                     cudaStream_t stream);

/*
 * skel_debug_grid_timeout -- launches `grid` co-resident CTAs on the grid-wide wait used by
 * the persistent pivot and QR kernels, with CTA 0 never arriving, so every other CTA gives up
 * after wait_ns nanoseconds (<= 5e9) and SKEL_ERR_TIMEOUT is written to dev_status.  Tests
 * the failure path without hanging the device.  Workspace handshake as elsewhere.
 */
skel_status skel_debug_grid_timeout(int grid, uint64_t wait_ns, void* ws, size_t* ws_bytes,
                                    int32_t* dev_status, cudaStream_t stream);

/*
 * skel_debug_fma_rate -- measurement aid (no counterpart in the paper): launches 8 CTAs per SM
 * of 256 threads, each thread running 8 independent FMA chains of `iters` steps in FP64
 * (fp64 != 0) or FP32, and writes the flop count of the launch to *flops (host).  The caller
 * times the launch with CUDA events on `stream`: flops / time is the FMA rate the pivot
 * solves and the float-float products are measured against.  sink: device buffer of at least
 * 8 x SMs elements of the type (never written in practice).
 */
skel_status skel_debug_fma_rate(int fp64, int64_t iters, int64_t* flops, void* sink, cudaStream_t stream);

/*
 * skel_debug_exchange_latency -- measurement aid (no counterpart in the paper): the time of one
 * round of the exchanges the pivoting kernels are built on, written to *ns_per_step (device
 * double) as the mean over rounds 1 .. steps-1 (globaltimer of CTA 0).
 *   kind 0: grid-wide barrier through global memory (the persistent LUPP / CPQR / QR kernels),
 *           `ctas` co-resident CTAs (2 .. SMs), cooperative launch; workspace (handshake).
 *   kind 1: candidate exchange in one thread-block cluster of `ctas` CTAs (2, 4, 8 or 16; 16
 *           needs the non-portable size, else SKEL_ERR_UNSUPPORTED): per round every CTA sends
 *           a 16-byte header and `col_words` (a multiple of 4, <= 64) 32-bit words to every CTA
 *           with st.async stores completing on three rotating mbarrier inboxes, as the LUPP
 *           panel kernel does per pivot step; no workspace (*ws_bytes = 0).
 * Waits are bounded (1 s, then SKEL_ERR_TIMEOUT in dev_status).  2 <= steps <= 10^6.
 */
skel_status skel_debug_exchange_latency(int kind, int ctas, int steps, int col_words, double* ns_per_step, void* ws,
                                        size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * skel_debug_kernel_timing -- measurement aid (no counterpart in the paper): enable != 0 makes
 * the launch sites of the hot kernels record a CUDA event on the launching stream before and
 * after each launch, from now on; enable == 0 stops recording.  Either call discards earlier
 * records.  Costs one branch per launch while disabled (the default).
 * skel_debug_kernel_time -- total device time (ms) and launch count of the recorded launches
 * of one kernel since the last skel_debug_kernel_timing call; waits for those launches.
 * Names: "sketch_tc", "sketch_fp8", "fp8_quantize", "gemm_tc" (W = Q^T A), "lupp_panel", "lupp_trail", "qr_panel", "qr_wy", "trsm",
 * "gemm_qr" (QR trailing updates and Q formation), "gemm_cur" (W Q_R), "gemm_eta_h" (R R^T),
 * "gemm_eta_sq" (eta's squarings), "gemm_refine" (the products of skel_id_refine), "gemm_simt" (other SIMT
 * GEMMs), "sparse_csc" (the CSC sparse-sign sketch), "batch_sketch", "batch_lupp", "batch_z",
 * "transpose" (A^T for the column and power sketches on the tensor cores).
 * Host-side state, process-wide; not for concurrent use from several threads.
 */
skel_status skel_debug_kernel_timing(int enable);
skel_status skel_debug_kernel_time(const char* kernel, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* SKEL_H */
