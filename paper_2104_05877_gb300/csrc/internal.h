// Host-side launchers shared between the translation units of libskel.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/skel.h"
#include "context_cache.h"

namespace skel {

// Strided view of an operand: element (r, c) at p[r*sr + c*sc].
struct View {
  const void* p;
  int64_t sr, sc;
};

enum GemmLeft { LEFT_LOAD = 0, LEFT_GAUSSIAN = 1 };
enum GemmEpi {
  EPI_STORE = 0,       // out(r,c) = alpha*acc
  EPI_STORE_SQ = 1,    // store, and partial[block] = sum (alpha*acc)^2
  EPI_RESID = 2,       // partial[block] = sum (ref(r,c) - alpha*acc)^2
  EPI_SKETCH = 3,      // store, flag non-finite outputs
  EPI_ACCUM = 4        // out(r,c) += alpha*acc (no K split)
};

// out(M x N) = alpha * L(M x K) * B(K x N).  `f64` selects FP64 storage+arithmetic for the
// operands (true) or FP32 (false); L/B/ref are converted on load from their own dtypes.
struct GemmArgs {
  int64_t M, N, K;
  View L;  skel_dtype l_dt;   // ignored for LEFT_GAUSSIAN
  View B;  skel_dtype b_dt;
  void* out; int64_t out_sr, out_sc; skel_dtype out_dt;
  View ref; skel_dtype ref_dt;     // EPI_RESID
  double alpha;
  double* partials;                // EPI_STORE_SQ / EPI_RESID: gemm_num_blocks(M, N) doubles
  uint64_t seed;                   // LEFT_GAUSSIAN
  int64_t gcol0 = 0;               // LEFT_GAUSSIAN: Gamma column of K index 0 (a multiple of 4)
  int32_t* dev_status;
  void* splitk_ws;                 // optional: gemm_workspace() bytes enable a K-split
  int64_t kchunk;                  // set by launch_gemm
  const char* timer = nullptr;     // kernel-timing name ("gemm_simt" when null)
};
int64_t gemm_num_blocks(int64_t M, int64_t N);
// Scratch for splitting K across CTAs when the M x N tiles cannot fill the GPU (STORE and
// STORE_SQ epilogues with a loaded left operand); 0 when no split is used.
size_t gemm_workspace(int64_t M, int64_t N, int64_t K, bool f64);
cudaError_t launch_gemm(const GemmArgs& a, bool f64, GemmLeft left, GemmEpi epi, cudaStream_t st);
// C += alpha A B for FP32 with 1 <= K <= 64: A (M x K) column-major, B (K x N) row-major, C
// (M x N) column-major (gemm_update.cu); `timer` names the launch for kernel timing.
cudaError_t launch_rank_update_f32(int64_t M, int64_t N, int K, const float* A, int64_t lda, const float* B,
                                   int64_t ldb, float* C, int64_t ldc, float alpha, const char* timer,
                                   cudaStream_t st);

// H = R R^T (s x s FP64, row-major ldh) for an FP32 s x n row-major R, float-float accumulation
// (~44 bits) on the FP32 pipes; workspace syrk_ff_workspace(s, n) bytes.
size_t syrk_ff_workspace(int32_t s, int64_t n);
cudaError_t launch_syrk_ff(int32_t s, int64_t n, const float* R, int64_t ldr, double* H, int64_t ldh, void* ws,
                           cudaStream_t st);
// Z(r, Js[t]) = delta(r, t) for an s x ? row-major FP64 Z.
cudaError_t launch_unit_columns(int32_t s, const int32_t* Js, double* Z, int64_t ldz, cudaStream_t st);
// Sum `count` doubles in `partials` (deterministic) into *out (device), optionally sqrt.
cudaError_t launch_reduce_sum(const double* partials, int64_t count, double* out, int take_sqrt,
                              cudaStream_t st);
// ||A||_F^2 of an m x n column-major matrix -> partials (one per block), returns #blocks.
int64_t sqnorm_num_blocks(int64_t m, int64_t n);
cudaError_t launch_sqnorm(int64_t m, int64_t n, skel_dtype dt, const void* A, int64_t lda,
                          double* partials, cudaStream_t st);

// The gathers write NaN for an index outside [0, ncols) (or [0, nrows)) and never read A there.
// C(:, r) = A(:, idx[r]) (m x s column-major out, ld = ldc) for A with ncols columns, dtype preserved.
cudaError_t launch_gather_cols(int64_t m, int32_t s, skel_dtype dt, const void* A, int64_t lda, int64_t ncols,
                               const int32_t* idx, void* C, int64_t ldc, cudaStream_t st);
// Rt(c, r) = A(idx[r], c) for A with nrows rows: the transpose of the row gather, n x s
// column-major (ld = ldr).
cudaError_t launch_gather_rows_t(int64_t n, int32_t s, skel_dtype dt, const void* A, int64_t lda, int64_t nrows,
                                 const int32_t* idx, void* Rt, int64_t ldr, cudaStream_t st);
// out(r, t) = F(r, idx[t]) for an s x ncols row-major F: s x s row-major FP64 out.
cudaError_t launch_gather_cols_rowmajor_f64(int32_t s, skel_dtype dt, const void* F, int64_t ldf, int64_t ncols,
                                            const int32_t* idx, double* out, int64_t ldo,
                                            cudaStream_t st);
// out = in^T for an s x s row-major FP64 matrix.
cudaError_t launch_transpose_f64(int32_t s, const double* in, int64_t ldi, double* out,
                                 int64_t ldo, cudaStream_t st);
// At = A^T for an m x n column-major FP32 A: At is n x m column-major (ld = ldt >= n).
cudaError_t launch_transpose_f32(int64_t m, int64_t n, const float* A, int64_t lda, float* At, int64_t ldt,
                                 cudaStream_t st);
// Set d[0..count) = value.
cudaError_t launch_fill_f64(double* d, int64_t count, double value, cudaStream_t st);

// Y = R^{-1} B for an s x s upper triangular FP64 R (row-major), B s x N row-major of dtype
// b_dt, Y s x N row-major FP64 (may alias B only when b_dt == SKEL_F64 and ldb == ldy).
cudaError_t launch_trsm_upper(int32_t s, int64_t N, const double* R, int64_t ldr, int unit_diag,
                              skel_dtype b_dt, const void* B, int64_t ldb, double* Y, int64_t ldy,
                              cudaStream_t st);

// Z = R^{-1} B for an FP32 right-hand side B (s x N row-major) in float-float arithmetic (R FP64
// upper triangular, split into float pairs in the workspace of trsm_ff_workspace(s) bytes).
size_t trsm_ff_workspace(int32_t s);
cudaError_t launch_trsm_upper_ff(int32_t s, int64_t N, const double* R, int64_t ldr, const float* B, int64_t ldb,
                                 double* Y, int64_t ldy, void* ws, cudaStream_t st);

// Y = R^{-T} D in place (D s x N row-major FP64, ldd) for an s x s upper triangular FP64 R,
// through U = J R^T J (s x s scratch) and the upper solve on the rows in reverse order.
cudaError_t launch_trsm_upper_t(int32_t s, int64_t N, const double* R, int64_t ldr, double* U, double* D,
                                int64_t ldd, cudaStream_t st);
// Z += X for s x n row-major FP64 (FP32) matrices.
cudaError_t launch_axpy_rows_f64(int32_t s, int64_t n, const double* X, int64_t ldx, double* Z, int64_t ldz,
                                 cudaStream_t st);
cudaError_t launch_axpy_rows_f32(int32_t s, int64_t n, const float* X, int64_t ldx, float* Z, int64_t ldz,
                                 cudaStream_t st);
// out = C^T B (s x n row-major FP64, ldo) for FP32 column-major C (m x s) and B (m x n): exact
// products, float-float sums (~44 bits); workspace gemm_tn_ff_workspace bytes.
size_t gemm_tn_ff_workspace(int64_t m, int64_t n, int32_t s);
cudaError_t launch_gemm_tn_ff(int64_t m, int64_t n, int32_t s, const float* C, int64_t ldc, const float* B,
                              int64_t ldb, double* out, int64_t ldo, void* ws, const char* timer, cudaStream_t st);

// sqrt(lambda_max(G)) for a symmetric positive definite s x s FP64 G (row-major): trace
// normalisation and repeated squaring, then power iteration in one CTA.  Writes *out.
size_t power_scratch_bytes(int32_t s);
cudaError_t launch_power_sqrt_lmax(int32_t s, const double* G, int64_t ldg, double* out,
                                   double* scratch /* power_scratch_bytes(s) */, cudaStream_t st);

// Persistent pivoting kernels (pivot.cu).
size_t lupp_workspace(skel_dtype dt, int64_t n, int32_t s, int* grid_out);
skel_status run_lupp(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s, int32_t* Js,
                     void* L, int64_t ldl, void* R, int64_t ldr, void* ws, size_t ws_bytes,
                     int32_t* dev_status, cudaStream_t st);
// LUPP through the panel-blocked cluster kernels when a panel fits one cluster's shared
// memory (lupp_panel.cu), else through the grid-barrier kernel above.
size_t lupp_auto_workspace(skel_dtype dt, int64_t n, int32_t s);
// Unique id of the calling thread's current CUDA context (cuCtxGetId), after making the
// current device's primary context current when the thread has none; 0 when the driver
// offers no context ids (context.cu).
unsigned long long current_context_id();

// Auxiliary stream and events for fork/join concurrency inside one call, one set per context
// and device (context_cache.h), created on first use.  Hold aux_mutex() for the whole enqueue that uses them, so that
// concurrent callers never interleave records and waits on the shared events.
constexpr int kAuxEvents = 130;      // one per panel of >= 8 steps of up to 1024, and spares
struct AuxSet {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t col[kAuxEvents] = {};
};
std::mutex& aux_mutex();
AuxSet* aux_set();
// Joins the auxiliary stream back into `st` when it goes out of scope, so that no return
// path (errors included) leaves work of the call running on the auxiliary stream unordered
// with the caller's stream.
struct AuxJoin {
  cudaStream_t st;
  AuxSet* aux;
  ~AuxJoin() {
    if (aux && cudaEventRecord(aux->join, aux->st) == cudaSuccess) cudaStreamWaitEvent(st, aux->join, 0);
  }
};

// Column LUPP on X and row LUPP on C^T (C = A(:, Js)) with the row chain pipelined behind the
// column chain on an auxiliary stream (lupp_panel.cu); usable when both fit the panel kernel.
bool skeleton_pivot_pipelined(skel_dtype dt, int64_t n, int64_t m, int32_t s);
size_t skeleton_pivot_workspace(skel_dtype dt, int64_t n, int64_t m, int32_t s);
skel_status run_skeleton_pivot(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s, const void* A,
                               int64_t m, int64_t lda, int32_t* Js, int32_t* Is, void* L, int64_t ldl, void* R,
                               int64_t ldr, void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t st);
skel_status run_lupp_auto(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s,
                          int32_t* Js, void* L, int64_t ldl, void* R, int64_t ldr, void* ws,
                          size_t ws_bytes, int32_t* dev_status, cudaStream_t st);
size_t cpqr_workspace(skel_dtype dt, int64_t l, int64_t n, int32_t s, int* grid_out);
skel_status run_cpqr(skel_dtype dt, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                     int32_t* Js, void* R, int64_t ldr, void* ws, size_t ws_bytes,
                     int32_t* dev_status, cudaStream_t st);

// Householder QR of a tall m x s column-major C (qr.cu): explicit Q (m x s col-major, same
// dtype, ld = ldq) and R (s x s row-major FP64).
// Panel-blocked Householder QR on thread-block clusters: reflectors V (m x s, unit lower
// trapezoidal, column-major), R (s x s row-major FP64) and, when Q is given, the explicit
// Q_C = H_0 .. H_{s-1} [I; 0] (m x s column-major).  qr_panels_workspace returns 0 and
// run_qr_panels SKEL_ERR_UNSUPPORTED when a panel of at least 8 columns does not fit a cluster.
size_t qr_panels_workspace(skel_dtype dt, int64_t m, int32_t s);
skel_status run_qr_panels(skel_dtype dt, const void* C, int64_t m, int64_t ldc, int32_t s, void* V,
                          int64_t ldv, double* R, int64_t ldr, void* Q, int64_t ldq, void* ws, size_t ws_bytes,
                          int32_t* dev_status, cudaStream_t st);
// W = Q^T A (s x n row-major FP32) on the tensor cores, 3xTF32 (FP32-level accuracy), for FP32
// Q (m x s) and A (m x n) column-major; sq_partials (optional) receives gemm_tc_num_partials
// partial sums of W^2 in a fixed order.
bool gemm_tc_usable(int64_t m, int64_t n, int32_t s, const void* Q, int64_t ldq, const void* A, int64_t lda);
size_t gemm_tc_workspace(int64_t m, int64_t n, int32_t s);
// An upper bound of gemm_tc_workspace(m', n', s) over every m' <= m and n' <= nmax.
size_t gemm_tc_workspace_bound(int64_t m, int64_t nmax, int32_t s);
int64_t gemm_tc_num_partials(int64_t m, int64_t n, int32_t s);
cudaError_t launch_gemm_tc_tn(int64_t m, int64_t n, int32_t s, const float* Q, int64_t ldq, const float* A,
                              int64_t lda, float* W, int64_t ldw, double* sq_partials, void* ws,
                              int32_t* dev_status, cudaStream_t st, const char* timer = "gemm_tc");
size_t qr_workspace(skel_dtype dt, int64_t m, int32_t s);
skel_status run_qr(skel_dtype dt, const void* C, int64_t m, int64_t ldc, int32_t s, void* Q,
                   int64_t ldq, double* R, int64_t ldr, void* ws, size_t ws_bytes,
                   int32_t* dev_status, cudaStream_t st);

// Sparse sign / CSC sketches (sparse.cu).
size_t sparse_pattern_bytes(int64_t m, int32_t zeta);
cudaError_t launch_sparse_pattern(int64_t row0, int64_t m, int32_t l, int32_t zeta, uint64_t seed,
                                  int32_t* table, cudaStream_t st);
cudaError_t launch_sparse_sketch_dense(int64_t m, int64_t n, skel_dtype dt, const void* A,
                                       int64_t lda, int32_t l, int32_t zeta,
                                       const int32_t* table, void* X, int64_t ldx,
                                       int32_t* dev_status, cudaStream_t st);
cudaError_t launch_sparse_sketch_csc(int64_t m, int64_t n, const int64_t* col_ptr,
                                     const int32_t* row_idx, const float* val, int32_t l,
                                     int32_t zeta, const int32_t* table, float* X, int64_t ldx,
                                     int32_t* dev_status, cudaStream_t st);
cudaError_t launch_gauss_sketch_csc(int64_t m, int64_t n, const int64_t* col_ptr,
                                    const int32_t* row_idx, const float* val, int32_t l,
                                    uint64_t seed, float* X, int64_t ldx, int32_t* dev_status,
                                    cudaStream_t st);

// Tensor-core Gaussian sketch (sketch_tc.cu).  Returns cudaErrorNotSupported when the
// shape or alignment is outside what the kernel handles.  ws: sketch_tc_workspace bytes.
size_t sketch_tc_workspace(int64_t m, int64_t n, int32_t l, skel_prec prec, bool srtt = false);
// FP8 (e4m3, per-128-row power-of-two scales) sketch (sketch_fp8.cu): quantisation pre-pass,
// e4m3 Gamma, tcgen05 kind::f8f6f4.  ws: sketch_fp8_workspace bytes.
size_t sketch_fp8_workspace(int64_t m, int64_t n, int32_t l);
cudaError_t launch_sketch_fp8(int64_t row0, int64_t m, int64_t n, const float* A, int64_t lda, int32_t l,
                              uint64_t seed, float* X, int64_t ldx, void* ws, int32_t* dev_status, cudaStream_t st);
// With srtt_tab / srtt_sel non-null (row0 = 0), Gamma is the SRTT's (srtt.cu tables) instead
// of the Gaussian's.
cudaError_t launch_sketch_tc(int64_t row0, int64_t m, int64_t n, const float* A, int64_t lda, int32_t l,
                             skel_prec prec, uint64_t seed, float* X, int64_t ldx, void* ws,
                             int32_t* dev_status, cudaStream_t st, const int32_t* srtt_tab = nullptr,
                             const int32_t* srtt_sel = nullptr);

// SRTT embedding (srtt.cu): tab (srtt_table_words(m) int32, 16-byte aligned) holds
// pi^{-1}(q) | (phi < 0) << 31 per column q of Gamma, sel the l selected rows; the dense
// Gamma * sqrt(l) (l x m row-major, ldg) for the SIMT GEMM.
uint64_t srtt_minv(int64_t m);
size_t srtt_table_words(int64_t m);
cudaError_t launch_srtt_tables(int64_t m, int32_t l, uint64_t seed, int32_t* tab, int32_t* sel, cudaStream_t st);
cudaError_t launch_srtt_dense(int64_t m, int32_t l, const int32_t* tab, const int32_t* sel, skel_dtype dt, void* G,
                              int64_t ldg, cudaStream_t st);

int device_sm_count();
// Number of kernels this library has launched in the process (diagnostics).
void note_launches(int n);

// CUDA events around one kernel launch (scope), recorded only while skel_debug_kernel_timing
// is enabled: construct immediately before the launch, destroy immediately after it.
bool kernel_timing_enabled();
class KernelTimer {
 public:
  KernelTimer(const char* name, cudaStream_t st);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  void* start_ = nullptr;
  void* stop_ = nullptr;
};
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

}  // namespace skel
