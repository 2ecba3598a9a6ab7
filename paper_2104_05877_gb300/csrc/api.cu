// C ABI entry points of libskel (include/skel.h): argument checks, workspace planning and
// stream-ordered launches.  No entry point allocates memory or synchronizes the host.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

#include <atomic>
#include <mutex>

using namespace skel;

namespace {

std::atomic<unsigned long long> g_launches{0};

// Carves 256-byte aligned regions out of the caller's workspace.  The same sequence of
// take() calls runs once to size the workspace (base == nullptr) and once to use it.
struct Arena {
  char* base;
  size_t off = 0;
  explicit Arena(void* b) : base(static_cast<char*>(b)) {}
  void* take(size_t bytes) {
    void* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  }
};

#define SK_CUDA(x)                                 \
  do {                                             \
    if ((x) != cudaSuccess) return SKEL_ERR_CUDA;  \
  } while (0)
#define SK_TRY(x)                      \
  do {                                 \
    skel_status _s = (x);              \
    if (_s != SKEL_OK) return _s;      \
  } while (0)

size_t esize(skel_dtype dt) { return dt == SKEL_F64 ? 8 : 4; }
bool valid_dtype(skel_dtype dt) { return dt == SKEL_F64 || dt == SKEL_F32; }

// Common workspace handshake: returns true when the call should stop here (size query or
// error); *st receives the status to return.
bool ws_handshake(size_t need, void* ws, size_t* ws_bytes, skel_status* st) {
  if (ws_bytes == nullptr) { *st = SKEL_ERR_INVALID_ARG; return true; }
  if (ws == nullptr) {
    *ws_bytes = need;
    *st = SKEL_OK;
    return true;
  }
  if (*ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    *st = SKEL_ERR_WORKSPACE;
    return true;
  }
  return false;
}

}  // namespace

void skel::note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

extern "C" {

uint64_t skel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* skel_status_string(int status) {
  switch (status) {
    case SKEL_OK: return "ok";
    case SKEL_ERR_INVALID_ARG: return "invalid argument";
    case SKEL_ERR_WORKSPACE: return "workspace too small or misaligned";
    case SKEL_ERR_NONFINITE: return "non-finite value in the data";
    case SKEL_ERR_RANK_DEFICIENT: return "zero pivot (rank deficient)";
    case SKEL_ERR_TIMEOUT: return "grid-wide wait timed out";
    case SKEL_ERR_CUDA: return "CUDA runtime error";
    case SKEL_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

int skel_version(void) { return 100; }

// ------------------------------------------------------------------------------------
skel_status skel_sketch(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda,
                        int32_t l, skel_sketch_kind kind, int32_t zeta, skel_prec prec,
                        uint64_t seed, void* X, int64_t ldx, void* ws, size_t* ws_bytes,
                        int32_t* dev_status, cudaStream_t stream) {
  return skel_sketch_rows(0, m, n, a_dtype, A, lda, l, kind, zeta, prec, seed, X, ldx, ws, ws_bytes, dev_status,
                          stream);
}

namespace {

// X = Gamma A for the SRTT (Sec. 2.3, item 2): the permutation / sign / selection tables,
// then the tensor-core kernel generating Gamma's tiles from them (TF32, BF16) or a dense
// Gamma and the SIMT GEMM (FP64, FP32).
skel_status sketch_srtt(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                        skel_prec prec, uint64_t seed, void* X, int64_t ldx, void* ws, size_t* ws_bytes,
                        int32_t* dev_status, cudaStream_t stream) {
  const bool tensor = prec == SKEL_PREC_TF32 || prec == SKEL_PREC_BF16;
  const skel_dtype x_dt = prec == SKEL_PREC_F64 ? SKEL_F64 : SKEL_F32;
  Arena ar(ws);
  int32_t* tab = static_cast<int32_t*>(ar.take(sizeof(int32_t) * srtt_table_words(m)));
  int32_t* sel = static_cast<int32_t*>(ar.take(sizeof(int32_t) * (size_t)l));
  void* G = !tensor ? ar.take(esize(x_dt) * (size_t)l * m) : nullptr;
  void* tcws = tensor && n > 0 ? ar.take(sketch_tc_workspace(m, n, l, prec, true)) : nullptr;
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  if (n == 0) return SKEL_OK;
  SK_CUDA(launch_srtt_tables(m, l, seed, tab, sel, stream));
  if (tensor) {
    const cudaError_t e = launch_sketch_tc(0, m, n, static_cast<const float*>(A), lda, l, prec, seed,
                                           static_cast<float*>(X), ldx, tcws, dev_status, stream, tab, sel);
    if (e == cudaErrorNotSupported) return SKEL_ERR_UNSUPPORTED;
    SK_CUDA(e);
    return SKEL_OK;
  }
  SK_CUDA(launch_srtt_dense(m, l, tab, sel, x_dt, G, m, stream));
  GemmArgs a{};
  a.M = l; a.N = n; a.K = m;
  a.L = View{G, m, 1}; a.l_dt = x_dt;
  a.B = View{A, 1, lda}; a.b_dt = a_dtype;
  a.out = X; a.out_sr = ldx; a.out_sc = 1; a.out_dt = x_dt;
  a.alpha = 1.0 / std::sqrt((double)l);
  a.dev_status = dev_status;
  SK_CUDA(launch_gemm(a, prec == SKEL_PREC_F64, LEFT_LOAD, EPI_SKETCH, stream));
  return SKEL_OK;
}

}  // namespace

skel_status skel_sketch_rows(int64_t row0, int64_t m, int64_t n, skel_dtype a_dtype, const void* A,
                             int64_t lda, int32_t l, skel_sketch_kind kind, int32_t zeta, skel_prec prec,
                             uint64_t seed, void* X, int64_t ldx, void* ws, size_t* ws_bytes,
                             int32_t* dev_status, cudaStream_t stream) {
  if (row0 < 0 || row0 % 4 != 0 || row0 + m > 0xFFFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || l < 1 || l > 4096 || !valid_dtype(a_dtype)) return SKEL_ERR_INVALID_ARG;
  if (lda < std::max<int64_t>(1, m) || ldx < std::max<int64_t>(1, n)) return SKEL_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && A == nullptr) || (n > 0 && X == nullptr)) return SKEL_ERR_INVALID_ARG;
  if (m > 0xFFFFFFFFll || n > 0xFFFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (prec < SKEL_PREC_F64 || prec > SKEL_PREC_FP8) return SKEL_ERR_INVALID_ARG;
  if (prec == SKEL_PREC_F64 && a_dtype != SKEL_F64) return SKEL_ERR_INVALID_ARG;
  if (kind != SKEL_SKETCH_GAUSSIAN && kind != SKEL_SKETCH_SPARSE_SIGN && kind != SKEL_SKETCH_SRTT)
    return SKEL_ERR_INVALID_ARG;
  const skel_dtype x_dt = prec == SKEL_PREC_F64 ? SKEL_F64 : SKEL_F32;
  if (kind == SKEL_SKETCH_SRTT) {
    if (l > m || m > (int64_t)INT32_MAX) return SKEL_ERR_INVALID_ARG;
    if (row0 != 0 || prec == SKEL_PREC_FP8) return SKEL_ERR_UNSUPPORTED;
    if (prec != SKEL_PREC_F64 && a_dtype != SKEL_F32) return SKEL_ERR_UNSUPPORTED;
    return sketch_srtt(m, n, a_dtype, A, lda, l, prec, seed, X, ldx, ws, ws_bytes, dev_status, stream);
  }
  Arena ar(ws);
  int32_t* table = nullptr;
  if (kind == SKEL_SKETCH_SPARSE_SIGN) {
    if (zeta < 1 || zeta > 31 || zeta > l) return SKEL_ERR_INVALID_ARG;
    if (prec == SKEL_PREC_TF32 || prec == SKEL_PREC_BF16 || prec == SKEL_PREC_FP8) return SKEL_ERR_UNSUPPORTED;
    if (esize(x_dt) * (size_t)l * 32 + 4 * 256 * (size_t)zeta > 220 * 1024) return SKEL_ERR_UNSUPPORTED;
    if (prec == SKEL_PREC_F32 && a_dtype != SKEL_F32) return SKEL_ERR_UNSUPPORTED;
    table = static_cast<int32_t*>(ar.take(sparse_pattern_bytes(m, zeta)));
  }
  const bool fp8 = kind == SKEL_SKETCH_GAUSSIAN && prec == SKEL_PREC_FP8;
  const bool tensor = kind == SKEL_SKETCH_GAUSSIAN && (prec == SKEL_PREC_BF16 || prec == SKEL_PREC_TF32 || fp8);
  if (tensor && a_dtype != SKEL_F32) return SKEL_ERR_UNSUPPORTED;
  if (fp8 && row0 != 0) return SKEL_ERR_UNSUPPORTED;
  void* tcws = tensor && m > 0 && n > 0
                   ? ar.take(fp8 ? sketch_fp8_workspace(m, n, l) : sketch_tc_workspace(m, n, l, prec))
                   : nullptr;
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  if (n == 0) return SKEL_OK;
  if (kind == SKEL_SKETCH_SPARSE_SIGN) {
    if (m == 0) {
      for (int32_t r = 0; r < l; ++r)
        SK_CUDA(cudaMemsetAsync(static_cast<char*>(X) + esize(x_dt) * r * ldx, 0, esize(x_dt) * n, stream));
      return SKEL_OK;
    }
    SK_CUDA(launch_sparse_pattern(row0, m, l, zeta, seed, table, stream));
    SK_CUDA(launch_sparse_sketch_dense(m, n, a_dtype, A, lda, l, zeta, table, X, ldx, dev_status, stream));
    return SKEL_OK;
  }
  if (tensor && m > 0) {
    const cudaError_t e =
        fp8 ? launch_sketch_fp8(row0, m, n, static_cast<const float*>(A), lda, l, seed, static_cast<float*>(X), ldx,
                                tcws, dev_status, stream)
            : launch_sketch_tc(row0, m, n, static_cast<const float*>(A), lda, l, prec, seed,
                               static_cast<float*>(X), ldx, tcws, dev_status, stream);
    if (e == cudaErrorNotSupported) return SKEL_ERR_UNSUPPORTED;
    SK_CUDA(e);
    return SKEL_OK;
  }
  GemmArgs a{};
  a.M = l; a.N = n; a.K = m;
  a.B = View{A, 1, lda}; a.b_dt = a_dtype;
  a.out = X; a.out_sr = ldx; a.out_sc = 1; a.out_dt = x_dt;
  a.alpha = 1.0 / std::sqrt((double)l);
  a.seed = seed;
  a.gcol0 = row0;
  a.dev_status = dev_status;
  SK_CUDA(launch_gemm(a, prec == SKEL_PREC_F64, LEFT_GAUSSIAN, EPI_SKETCH, stream));
  return SKEL_OK;
}

}  // extern "C"

namespace {

// The copy stream and events of skel_sketch_host, one set per context and device
// (context_cache.h), created on first use.  copied[b] marks staging buffer b filled,
// consumed[b] the sketch of it finished.
struct HostStreamSet {
  cudaStream_t copy = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
};

std::mutex& host_stream_mutex() {
  static std::mutex mu;
  return mu;
}

HostStreamSet* host_stream_set() {
  static ContextCache<HostStreamSet> sets;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  return sets.get(current_context_id(), dev, [](HostStreamSet& h) {
    bool ok = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&h.fork, &h.join, &h.copied[0], &h.copied[1], &h.consumed[0], &h.consumed[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
  });
}

// Joins the copy stream back into the caller's stream on every return path.
struct HostStreamJoin {
  cudaStream_t st;
  HostStreamSet* h;
  ~HostStreamJoin() {
    if (cudaEventRecord(h->join, h->copy) == cudaSuccess) cudaStreamWaitEvent(st, h->join, 0);
  }
};

// Columns per panel: the caller's choice, else about 512 MiB of A: a multiple of 256 columns,
// of 4 for taller columns, and at least one column.
int64_t host_panel_cols(int64_t m, int64_t n, skel_dtype dt, int64_t panel) {
  if (panel > 0) return std::min(panel, n);
  int64_t w = ((int64_t)512 << 20) / std::max<int64_t>(1, (int64_t)esize(dt) * m);
  w = w >= 256 ? w / 256 * 256 : w >= 4 ? w / 4 * 4 : std::max<int64_t>(1, w);
  return std::min(w, n);
}

// Streams the column panels of A (w columns each; host or device memory) through the staging
// buffers stage[0..1] (leading dimension lds) and calls work(i, stage, j0, wi) on `stream` for
// panel i once its copy has landed; the copy of panel i + 1 runs meanwhile on the copy stream,
// and the copy of panel i + 2 waits until the work on panel i has finished with its buffer.
template <typename Work>
skel_status stream_panels(int64_t m, int64_t n, size_t ea, const void* A, int64_t lda, int64_t lds, int64_t w,
                          char* const stage[2], cudaStream_t stream, Work&& work) {
  std::lock_guard<std::mutex> lock(host_stream_mutex());
  HostStreamSet* h = host_stream_set();
  if (h == nullptr) return SKEL_ERR_CUDA;
  SK_CUDA(cudaEventRecord(h->fork, stream));
  SK_CUDA(cudaStreamWaitEvent(h->copy, h->fork, 0));
  HostStreamJoin joiner{stream, h};
  const int64_t npan = (n + w - 1) / w;
  for (int64_t i = 0; i < npan; ++i) {
    const int b = (int)(i & 1);
    const int64_t j0 = i * w, wi = std::min(w, n - j0);
    if (i >= 2) SK_CUDA(cudaStreamWaitEvent(h->copy, h->consumed[b], 0));
    const char* src = static_cast<const char*>(A) + ea * (size_t)lda * j0;
    if (lda == lds)   // contiguous columns: one linear copy
      SK_CUDA(cudaMemcpyAsync(stage[b], src, ea * (size_t)lds * (wi - 1) + ea * m, cudaMemcpyDefault, h->copy));
    else
      SK_CUDA(cudaMemcpy2DAsync(stage[b], ea * lds, src, ea * lda, ea * m, wi, cudaMemcpyDefault, h->copy));
    SK_CUDA(cudaEventRecord(h->copied[b], h->copy));
    SK_CUDA(cudaStreamWaitEvent(stream, h->copied[b], 0));
    SK_TRY(work(i, stage[b], j0, wi));
    SK_CUDA(cudaEventRecord(h->consumed[b], stream));
  }
  return SKEL_OK;
}

}  // namespace

extern "C" {

skel_status skel_sketch_host(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                             skel_sketch_kind kind, int32_t zeta, skel_prec prec, uint64_t seed, void* X,
                             int64_t ldx, int64_t panel, void* ws, size_t* ws_bytes, int32_t* dev_status,
                             cudaStream_t stream) {
  if (m < 0 || n < 0 || panel < 0 || !valid_dtype(a_dtype)) return SKEL_ERR_INVALID_ARG;
  if (lda < std::max<int64_t>(1, m) || ldx < std::max<int64_t>(1, n)) return SKEL_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && A == nullptr) || (n > 0 && X == nullptr)) return SKEL_ERR_INVALID_ARG;
  const skel_dtype x_dt = prec == SKEL_PREC_F64 ? SKEL_F64 : SKEL_F32;
  const int64_t w = n > 0 ? host_panel_cols(m, n, a_dtype, panel) : 0;
  const int64_t npan = w > 0 ? (n + w - 1) / w : 0;
  const int64_t wlast = npan > 0 ? n - (npan - 1) * w : 0;
  const int64_t lds = std::max<int64_t>(4, (m + 3) / 4 * 4);   // staging columns start 16-byte aligned
  // the sketch workspace of the two panel widths that occur (argument checks happen here too)
  size_t need_w = 0, need_last = 0;
  SK_TRY(skel_sketch_rows(0, m, w, a_dtype, A, lds, l, kind, zeta, prec, seed, X, ldx, nullptr, &need_w, dev_status,
                          stream));
  if (wlast > 0 && wlast != w)
    SK_TRY(skel_sketch_rows(0, m, wlast, a_dtype, A, lds, l, kind, zeta, prec, seed, X, ldx, nullptr, &need_last,
                            dev_status, stream));
  Arena ar(ws);
  char* stage[2];
  stage[0] = static_cast<char*>(m > 0 && n > 0 ? ar.take(esize(a_dtype) * (size_t)lds * w) : nullptr);
  stage[1] = static_cast<char*>(m > 0 && npan > 1 ? ar.take(esize(a_dtype) * (size_t)lds * w) : nullptr);
  size_t sws_bytes = std::max(need_w, need_last);
  void* sws = ar.take(sws_bytes);
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  if (n == 0) return SKEL_OK;
  if (m == 0) return skel_sketch_rows(0, 0, n, a_dtype, nullptr, lda, l, kind, zeta, prec, seed, X, ldx, sws,
                                      &sws_bytes, dev_status, stream);
  return stream_panels(m, n, esize(a_dtype), A, lda, lds, w, stage, stream,
                       [&](int64_t, const char* panel_a, int64_t j0, int64_t wi) -> skel_status {
                         size_t sz = sws_bytes;
                         return skel_sketch_rows(0, m, wi, a_dtype, panel_a, lds, l, kind, zeta, prec, seed,
                                                 static_cast<char*>(X) + esize(x_dt) * j0, ldx, sws, &sz,
                                                 dev_status, stream);
                       });
}

skel_status skel_sketch_host_two_sided(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda,
                                       int32_t l, skel_prec prec, uint64_t seed_gamma, uint64_t seed_omega, void* X,
                                       int64_t ldx, void* Yt, int64_t ldy, int64_t panel, void* ws, size_t* ws_bytes,
                                       int32_t* dev_status, cudaStream_t stream) {
  if (m < 1 || n < 1 || l < 1 || l > 4096 || !valid_dtype(a_dtype) || A == nullptr || X == nullptr ||
      Yt == nullptr || lda < m || ldx < n || ldy < m || panel < 0 || panel % 4 != 0 || n > 0xFFFFFFFFll)
    return SKEL_ERR_INVALID_ARG;
  if (prec == SKEL_PREC_FP8) return SKEL_ERR_UNSUPPORTED;
  if ((prec == SKEL_PREC_F64) != (a_dtype == SKEL_F64)) return SKEL_ERR_INVALID_ARG;
  const bool tc = prec == SKEL_PREC_TF32 || prec == SKEL_PREC_BF16;
  if (tc && m > (int64_t)INT32_MAX) return SKEL_ERR_UNSUPPORTED;
  const bool f64 = prec == SKEL_PREC_F64;
  const skel_dtype x_dt = f64 ? SKEL_F64 : SKEL_F32;
  const size_t ex = esize(x_dt), ea = esize(a_dtype);
  // panel offsets stay multiples of 4: Omega's counters take its columns four at a time
  const int64_t w = std::max<int64_t>(4, host_panel_cols(m, n, a_dtype, panel) / 4 * 4);
  const int64_t npan = (n + w - 1) / w;
  const int64_t wlast = n - (npan - 1) * w;
  const int64_t lds = (m + 3) / 4 * 4;
  const int64_t w4 = (w + 3) / 4 * 4;
  size_t need_w = 0, need_last = 0;
  SK_TRY(skel_sketch_rows(0, m, std::min(w, n), a_dtype, A, lds, l, SKEL_SKETCH_GAUSSIAN, 0, prec, seed_gamma, X,
                          ldx, nullptr, &need_w, dev_status, stream));
  if (wlast != w)
    SK_TRY(skel_sketch_rows(0, m, wlast, a_dtype, A, lds, l, SKEL_SKETCH_GAUSSIAN, 0, prec, seed_gamma, X, ldx,
                            nullptr, &need_last, dev_status, stream));
  size_t yws_bytes = tc ? std::max(sketch_tc_workspace(std::min(w, n), m, l, prec), sketch_tc_workspace(wlast, m, l, prec))
                        : std::max(gemm_workspace(l, m, std::min(w, n), f64), gemm_workspace(l, m, wlast, f64));
  Arena ar(ws);
  char* stage[2];
  stage[0] = static_cast<char*>(ar.take(ea * (size_t)lds * w));
  stage[1] = static_cast<char*>(npan > 1 ? ar.take(ea * (size_t)lds * w) : nullptr);
  size_t xws_bytes = std::max(need_w, need_last);
  void* xws = ar.take(xws_bytes);
  float* At = tc ? static_cast<float*>(ar.take(sizeof(float) * (size_t)w4 * m)) : nullptr;
  void* yws = ar.take(yws_bytes);
  char* part = static_cast<char*>(npan > 1 ? ar.take(ex * (size_t)l * m) : nullptr);
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  return stream_panels(m, n, ea, A, lda, lds, w, stage, stream,
                       [&](int64_t i, const char* panel_a, int64_t j0, int64_t wi) -> skel_status {
    // X(:, j0 : j0 + wi) = Gamma A(:, panel)   (Algorithm 3, row sketch)
    size_t sz = xws_bytes;
    SK_TRY(skel_sketch_rows(0, m, wi, a_dtype, panel_a, lds, l, SKEL_SKETCH_GAUSSIAN, 0, prec, seed_gamma,
                            static_cast<char*>(X) + ex * j0, ldx, xws, &sz, dev_status, stream));
    // Y^T += Omega(:, panel) A(:, panel)^T   (Algorithm 3, column sketch): the first
    // panel writes Y^T, later ones a partial that is added to it
    void* out = i == 0 ? Yt : part;
    const int64_t ldo = i == 0 ? ldy : m;
    if (tc) {
      SK_CUDA(launch_transpose_f32(m, wi, reinterpret_cast<const float*>(panel_a), lds, At, w4, stream));
      const cudaError_t e = launch_sketch_tc(j0, wi, m, At, w4, l, prec, seed_omega, static_cast<float*>(out), ldo,
                                             yws, dev_status, stream);
      if (e == cudaErrorNotSupported) return SKEL_ERR_UNSUPPORTED;
      SK_CUDA(e);
    } else {
      GemmArgs a{};
      a.M = l; a.N = m; a.K = wi;
      a.B = View{panel_a, lds, 1}; a.b_dt = a_dtype;      // B(k, c) = A(c, j0 + k)
      a.out = out; a.out_sr = ldo; a.out_sc = 1; a.out_dt = x_dt;
      a.alpha = 1.0 / std::sqrt((double)l);
      a.seed = seed_omega;
      a.gcol0 = j0;
      a.dev_status = dev_status;
      a.splitk_ws = yws;
      SK_CUDA(launch_gemm(a, f64, LEFT_GAUSSIAN, EPI_SKETCH, stream));
    }
    if (i > 0) {
      if (f64)
        SK_CUDA(launch_axpy_rows_f64(l, m, reinterpret_cast<const double*>(part), m, static_cast<double*>(Yt), ldy,
                                     stream));
      else
        SK_CUDA(launch_axpy_rows_f32(l, m, reinterpret_cast<const float*>(part), m, static_cast<float*>(Yt), ldy,
                                     stream));
    }
    return SKEL_OK;
  });
}

skel_status skel_sketch_cols(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                             skel_prec prec, uint64_t seed, void* Yt, int64_t ldy, void* ws, size_t* ws_bytes,
                             int32_t* dev_status, cudaStream_t stream) {
  if (m < 1 || n < 1 || l < 1 || l > 4096 || !valid_dtype(a_dtype) || A == nullptr || Yt == nullptr || lda < m ||
      ldy < m || n > 0xFFFFFFFFll)
    return SKEL_ERR_INVALID_ARG;
  if (prec == SKEL_PREC_FP8) return SKEL_ERR_UNSUPPORTED;
  if ((prec == SKEL_PREC_F64) != (a_dtype == SKEL_F64)) return SKEL_ERR_INVALID_ARG;
  if (prec == SKEL_PREC_TF32 || prec == SKEL_PREC_BF16) {
    // the tensor-core sketch on a transposed copy (A^T, n x m column-major): its K dimension
    // (A's columns) must be contiguous, and Omega's counters are those of the SIMT path
    if (m > (int64_t)INT32_MAX) return SKEL_ERR_UNSUPPORTED;
    const int64_t n4 = (n + 3) / 4 * 4;
    Arena ar(ws);
    float* At = static_cast<float*>(ar.take(sizeof(float) * (size_t)n4 * m));
    void* tcws = ar.take(sketch_tc_workspace(n, m, l, prec));
    skel_status st;
    if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
    SK_CUDA(launch_transpose_f32(m, n, static_cast<const float*>(A), lda, At, n4, stream));
    const cudaError_t e = launch_sketch_tc(0, n, m, At, n4, l, prec, seed, static_cast<float*>(Yt), ldy, tcws,
                                           dev_status, stream);
    if (e == cudaErrorNotSupported) return SKEL_ERR_UNSUPPORTED;
    SK_CUDA(e);
    return SKEL_OK;
  }
  const bool f64 = prec == SKEL_PREC_F64;
  Arena ar(ws);
  void* kws = ar.take(gemm_workspace(l, m, n, f64));
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  GemmArgs a{};
  a.M = l; a.N = m; a.K = n;
  a.B = View{A, lda, 1}; a.b_dt = a_dtype;            // B(k, c) = A^T(k, c) = A(c, k)
  a.out = Yt; a.out_sr = ldy; a.out_sc = 1; a.out_dt = f64 ? SKEL_F64 : SKEL_F32;
  a.alpha = 1.0 / std::sqrt((double)l);
  a.seed = seed;
  a.dev_status = dev_status;
  a.splitk_ws = kws;
  SK_CUDA(launch_gemm(a, f64, LEFT_GAUSSIAN, EPI_SKETCH, stream));
  return SKEL_OK;
}

skel_status skel_sketch_power(int64_t m, int64_t n, skel_dtype a_dtype, const void* A, int64_t lda, int32_t l,
                              int32_t q, skel_prec prec, uint64_t seed, void* X, int64_t ldx, void* ws,
                              size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (m < 1 || n < 1 || l < 1 || l > 4096 || q < 1 || q > 8 || !valid_dtype(a_dtype) || A == nullptr ||
      X == nullptr || lda < m || ldx < n || n > 0xFFFFFFFFll)
    return SKEL_ERR_INVALID_ARG;
  if (prec != SKEL_PREC_F64 && prec != SKEL_PREC_F32 && prec != SKEL_PREC_TF32) return SKEL_ERR_UNSUPPORTED;
  if ((prec == SKEL_PREC_F64) != (a_dtype == SKEL_F64)) return SKEL_ERR_INVALID_ARG;
  const bool f64 = prec == SKEL_PREC_F64;
  const skel_dtype dt = f64 ? SKEL_F64 : SKEL_F32;
  const bool tcw = !f64 && gemm_tc_usable(m, n, l, nullptr, m, A, lda);
  if (prec == SKEL_PREC_TF32 && tcw && m <= (int64_t)INT32_MAX) {
    // tensor cores throughout, on A and a transposed copy A^T (n x m column-major):
    // Y^T = Omega A^T by the TF32 sketch kernel (Omega generated), then X = Y^T A and, for
    // further iterations, Y^T = X A^T by the 3xTF32 GEMM
    const int64_t n4 = (n + 3) / 4 * 4;
    Arena ar(ws);
    float* At = static_cast<float*>(ar.take(sizeof(float) * (size_t)n4 * m));
    float* Ytf = static_cast<float*>(ar.take(sizeof(float) * (size_t)l * m));
    void* tcws = ar.take(sketch_tc_workspace(n, m, l, prec));
    void* kx = ar.take(gemm_tc_workspace(m, n, l));
    void* ky = ar.take(q > 1 ? gemm_tc_workspace(n, m, l) : 0);
    skel_status st;
    if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
    float* Xf = static_cast<float*>(X);
    SK_CUDA(launch_transpose_f32(m, n, static_cast<const float*>(A), lda, At, n4, stream));
    for (int it = 0; it < q; ++it) {
      if (it == 0) {
        const cudaError_t e = launch_sketch_tc(0, n, m, At, n4, l, prec, seed, Ytf, m, tcws, dev_status, stream);
        if (e == cudaErrorNotSupported) return SKEL_ERR_UNSUPPORTED;
        SK_CUDA(e);
      } else {
        SK_CUDA(launch_gemm_tc_tn(n, m, l, Xf, ldx, At, n4, Ytf, m, nullptr, ky, dev_status, stream));
      }
      SK_CUDA(launch_gemm_tc_tn(m, n, l, Ytf, m, static_cast<const float*>(A), lda, Xf, ldx, nullptr, kx,
                                dev_status, stream));
    }
    return SKEL_OK;
  }
  Arena ar(ws);
  void* Yt = ar.take(esize(dt) * (size_t)l * m);                  // Y^T = X_prev A^T, l x m row-major
  void* kws1 = ar.take(gemm_workspace(l, m, n, f64));
  void* kws2 = ar.take(tcw ? gemm_tc_workspace(m, n, l) : gemm_workspace(l, n, m, f64));
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  for (int it = 0; it < q; ++it) {
    // Y^T = Omega A^T (it = 0, Omega generated in the kernel, N(0, 1/l)) or X A^T
    GemmArgs a{};
    a.M = l; a.N = m; a.K = n;
    a.B = View{A, lda, 1}; a.b_dt = a_dtype;          // B(k, c) = A^T(k, c) = A(c, k)
    a.out = Yt; a.out_sr = m; a.out_sc = 1; a.out_dt = dt;
    a.dev_status = dev_status;
    a.splitk_ws = kws1;
    if (it == 0) {
      a.alpha = 1.0 / std::sqrt((double)l);
      a.seed = seed;
      SK_CUDA(launch_gemm(a, f64, LEFT_GAUSSIAN, EPI_SKETCH, stream));
    } else {
      a.L = View{X, ldx, 1}; a.l_dt = dt;
      a.alpha = 1.0;
      SK_CUDA(launch_gemm(a, f64, LEFT_LOAD, EPI_STORE, stream));
    }
    // X = Y^T A
    if (tcw) {
      SK_CUDA(launch_gemm_tc_tn(m, n, l, static_cast<const float*>(Yt), m, static_cast<const float*>(A), lda,
                                static_cast<float*>(X), ldx, nullptr, kws2, dev_status, stream));
    } else {
      GemmArgs b{};
      b.M = l; b.N = n; b.K = m;
      b.L = View{Yt, m, 1}; b.l_dt = dt;
      b.B = View{A, 1, lda}; b.b_dt = a_dtype;
      b.out = X; b.out_sr = ldx; b.out_sc = 1; b.out_dt = dt;
      b.alpha = 1.0;
      b.dev_status = dev_status;
      b.splitk_ws = kws2;
      SK_CUDA(launch_gemm(b, f64, LEFT_LOAD, EPI_STORE, stream));
    }
  }
  return SKEL_OK;
}

skel_status skel_sketch_csc(int64_t m, int64_t n, int64_t nnz, const int64_t* col_ptr,
                            const int32_t* row_idx, const float* val, int32_t l,
                            skel_sketch_kind kind, int32_t zeta, uint64_t seed, float* X,
                            int64_t ldx, void* ws, size_t* ws_bytes, int32_t* dev_status,
                            cudaStream_t stream) {
  if (m < 0 || n < 0 || nnz < 0 || l < 1 || l > 4096) return SKEL_ERR_INVALID_ARG;
  if (m > 0x7FFFFFFFll || n > 0xFFFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (ldx < std::max<int64_t>(1, n) || (n > 0 && (X == nullptr || col_ptr == nullptr)))
    return SKEL_ERR_INVALID_ARG;
  if (nnz > 0 && (row_idx == nullptr || val == nullptr)) return SKEL_ERR_INVALID_ARG;
  Arena ar(ws);
  int32_t* table = nullptr;
  if (kind == SKEL_SKETCH_SPARSE_SIGN) {
    if (zeta < 1 || zeta > 31 || zeta > l) return SKEL_ERR_INVALID_ARG;
    if (sizeof(float) * (size_t)l * 32 > 220 * 1024) return SKEL_ERR_UNSUPPORTED;
    table = static_cast<int32_t*>(ar.take(sparse_pattern_bytes(m, zeta)));
  } else if (kind != SKEL_SKETCH_GAUSSIAN) {
    return SKEL_ERR_INVALID_ARG;
  }
  skel_status st;
  if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
  if (n == 0) return SKEL_OK;
  if (kind == SKEL_SKETCH_SPARSE_SIGN) {
    SK_CUDA(launch_sparse_pattern(0, m, l, zeta, seed, table, stream));
    SK_CUDA(launch_sparse_sketch_csc(m, n, col_ptr, row_idx, val, l, zeta, table, X, ldx, dev_status, stream));
  } else {
    SK_CUDA(launch_gauss_sketch_csc(m, n, col_ptr, row_idx, val, l, seed, X, ldx, dev_status, stream));
  }
  return SKEL_OK;
}

// ------------------------------------------------------------------------------------
skel_status skel_pivot_lupp(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx,
                            int32_t s, int32_t* Js, void* L, int64_t ldl, void* R, int64_t ldr,
                            void* ws, size_t* ws_bytes, int32_t* dev_status,
                            cudaStream_t stream) {
  if (!valid_dtype(dtype) || X == nullptr || Js == nullptr) return SKEL_ERR_INVALID_ARG;
  if (s < 1 || s > kMaxS || s > l || s > n || n > 0x7FFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (ldx < n || (L && ldl < s) || (R && ldr < n)) return SKEL_ERR_INVALID_ARG;
  const size_t need = lupp_auto_workspace(dtype, n, s);
  skel_status st;
  if (ws_handshake(need, ws, ws_bytes, &st)) return st;
  return run_lupp_auto(dtype, X, n, ldx, s, Js, L, ldl, R, ldr, ws, *ws_bytes, dev_status, stream);
}

skel_status skel_pivot_skeleton(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                                const void* A, int64_t m, int64_t lda, int32_t* Js, int32_t* Is, void* L,
                                int64_t ldl, void* R, int64_t ldr, void* ws, size_t* ws_bytes, int32_t* dev_status,
                                cudaStream_t stream) {
  if (!valid_dtype(dtype) || X == nullptr || Js == nullptr || Is == nullptr || A == nullptr)
    return SKEL_ERR_INVALID_ARG;
  if (s < 1 || s > kMaxS || s > l || s > n || s > m || n > 0x7FFFFFFFll || m > 0x7FFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (ldx < n || lda < m || (L && ldl < s) || (R && ldr < n)) return SKEL_ERR_INVALID_ARG;
  if (skeleton_pivot_pipelined(dtype, n, m, s)) {
    const size_t need = skeleton_pivot_workspace(dtype, n, m, s);
    skel_status st;
    if (ws_handshake(need, ws, ws_bytes, &st)) return st;
    return run_skeleton_pivot(dtype, X, n, ldx, s, A, m, lda, Js, Is, L, ldl, R, ldr, ws, *ws_bytes, dev_status,
                              stream);
  }
  // one after the other: LUPP on X, then on C^T with C = A(:, Js)
  const size_t lc = lupp_auto_workspace(dtype, n, s), lr = lupp_auto_workspace(dtype, m, s);
  const size_t cbytes = align_up(esize(dtype) * (size_t)m * s);
  skel_status st;
  if (ws_handshake(std::max(lc, cbytes + lr), ws, ws_bytes, &st)) return st;
  SK_TRY(run_lupp_auto(dtype, X, n, ldx, s, Js, L, ldl, R, ldr, ws, *ws_bytes, dev_status, stream));
  void* C = ws;
  SK_CUDA(launch_gather_cols(m, s, dtype, A, lda, n, Js, C, m, stream));
  return run_lupp_auto(dtype, C, m, m, s, Is, nullptr, 0, nullptr, 0, static_cast<char*>(ws) + cbytes, lr, dev_status,
                       stream);
}

skel_status skel_pivot_cpqr(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx,
                            int32_t s, int32_t* Js, void* R, int64_t ldr, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!valid_dtype(dtype) || X == nullptr || Js == nullptr) return SKEL_ERR_INVALID_ARG;
  if (s < 1 || l > kMaxS || s > l || s > n || n > 0x7FFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (ldx < n || (R && ldr < n)) return SKEL_ERR_INVALID_ARG;
  const size_t need = cpqr_workspace(dtype, l, n, s, nullptr);
  skel_status st;
  if (ws_handshake(need, ws, ws_bytes, &st)) return st;
  return run_cpqr(dtype, X, l, n, ldx, s, Js, R, ldr, ws, *ws_bytes, dev_status, stream);
}

// ------------------------------------------------------------------------------------
namespace {

bool id_args_ok(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                const int32_t* Js) {
  return valid_dtype(dtype) && A && Js && m >= 1 && n >= 1 && s >= 1 && s <= kMaxS && s <= m &&
         s <= n && lda >= m;
}

// C = A(:, Js) (A: m x n); C = Q R.  Returns device pointers through the arena.
skel_status skeleton_qr(Arena& ar, bool run, int64_t m, int64_t n, skel_dtype dt, const void* A, int64_t lda,
                        int32_t s, const int32_t* idx, void** C, void** Q, double** R,
                        int32_t* dev_status, cudaStream_t st) {
  *C = ar.take(esize(dt) * (size_t)m * s);
  *Q = ar.take(esize(dt) * (size_t)m * s);
  *R = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
  const size_t qn = qr_workspace(dt, m, s);
  void* qws = ar.take(qn);
  if (!run) return SKEL_OK;
  SK_CUDA(launch_gather_cols(m, s, dt, A, lda, n, idx, *C, m, st));
  return run_qr(dt, *C, m, m, s, *Q, m, *R, s, qws, qn, dev_status, st);
}

}  // namespace

skel_status skel_id(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                    int32_t s, const int32_t* Js, double* Z, int64_t ldz, double* sq_norms,
                    void* ws, size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Z == nullptr || ldz < n) return SKEL_ERR_INVALID_ARG;
  const bool f64 = dtype == SKEL_F64;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void *C, *Q;
    double* R;
    SK_TRY(skeleton_qr(ar, run, m, n, dtype, A, lda, s, Js, &C, &Q, &R, dev_status, stream));
    void* W = ar.take(esize(dtype) * (size_t)s * n);
    const bool tcw = !f64 && gemm_tc_usable(m, n, s, nullptr, m, A, lda);   // tensor-core W
    const int64_t nbw = tcw ? gemm_tc_num_partials(m, n, s) : gemm_num_blocks(s, n);
    double* pw = static_cast<double*>(ar.take(sizeof(double) * nbw));
    const int64_t nba = sqnorm_num_blocks(m, n);
    double* pa = static_cast<double*>(ar.take(sizeof(double) * nba));
    void* kws = ar.take(tcw ? gemm_tc_workspace(m, n, s) : gemm_workspace(s, n, m, f64));
    void* tws = f64 ? nullptr : ar.take(trsm_ff_workspace(s));
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    GemmArgs g{};
    g.splitk_ws = kws;
    g.M = s; g.N = n; g.K = m;
    g.L = View{Q, m, 1}; g.l_dt = dtype;          // Q^T(r, i) = Q(i, r)
    g.B = View{A, 1, lda}; g.b_dt = dtype;
    g.out = W; g.out_sr = n; g.out_sc = 1; g.out_dt = dtype;
    g.alpha = 1.0;
    g.partials = pw;
    if (tcw)
      SK_CUDA(launch_gemm_tc_tn(m, n, s, static_cast<const float*>(Q), m, static_cast<const float*>(A), lda,
                                static_cast<float*>(W), n, pw, kws, dev_status, stream));
    else
      SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_STORE_SQ, stream));
    if (f64)
      SK_CUDA(launch_trsm_upper(s, n, R, s, 0, dtype, W, n, Z, ldz, stream));
    else    // the FP32 W in float-float arithmetic (FP32 pipes)
      SK_CUDA(launch_trsm_upper_ff(s, n, R, s, static_cast<const float*>(W), n, Z, ldz, tws, stream));
    if (sq_norms) {
      SK_CUDA(launch_sqnorm(m, n, dtype, A, lda, pa, stream));
      SK_CUDA(launch_reduce_sum(pa, nba, sq_norms, 0, stream));
      SK_CUDA(launch_reduce_sum(pw, nbw, sq_norms + 1, 0, stream));
    }
  }
  return SKEL_OK;
}

skel_status skel_id_refine(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                           int32_t s, const int32_t* Js, double* Z, int64_t ldz, double* sq_norms,
                           void* ws, size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Z == nullptr || ldz < n) return SKEL_ERR_INVALID_ARG;
  if (dtype != SKEL_F32) return SKEL_ERR_UNSUPPORTED;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void *C, *Q;
    double* R;
    SK_TRY(skeleton_qr(ar, run, m, n, dtype, A, lda, s, Js, &C, &Q, &R, dev_status, stream));
    void* W = ar.take(sizeof(float) * (size_t)s * n);
    const bool tcw = gemm_tc_usable(m, n, s, nullptr, m, A, lda);
    const int64_t nbw = tcw ? gemm_tc_num_partials(m, n, s) : gemm_num_blocks(s, n);
    double* pw = static_cast<double*>(ar.take(sizeof(double) * nbw));
    const int64_t nba = sqnorm_num_blocks(m, n);
    double* pa = static_cast<double*>(ar.take(sizeof(double) * nba));
    void* kws = ar.take(tcw ? gemm_tc_workspace(m, n, s) : gemm_workspace(s, n, m, false));
    double* D = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * n));     // C^T A, then the correction
    double* G = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));     // C^T C
    double* U = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));     // J R^T J
    void* fws = ar.take(std::max(gemm_tn_ff_workspace(m, n, s), gemm_tn_ff_workspace(m, s, s)));
    void* tws = ar.take(trsm_ff_workspace(s));
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    // Z0 = R_C^{-1} Q_C^T A, as skel_id
    if (tcw) {
      SK_CUDA(launch_gemm_tc_tn(m, n, s, static_cast<const float*>(Q), m, static_cast<const float*>(A), lda,
                                static_cast<float*>(W), n, pw, kws, dev_status, stream));
    } else {
      GemmArgs g{};
      g.splitk_ws = kws;
      g.M = s; g.N = n; g.K = m;
      g.L = View{Q, m, 1}; g.l_dt = dtype;
      g.B = View{A, 1, lda}; g.b_dt = dtype;
      g.out = W; g.out_sr = n; g.out_sc = 1; g.out_dt = dtype;
      g.alpha = 1.0;
      g.partials = pw;
      SK_CUDA(launch_gemm(g, false, LEFT_LOAD, EPI_STORE_SQ, stream));
    }
    SK_CUDA(launch_trsm_upper_ff(s, n, R, s, static_cast<const float*>(W), n, Z, ldz, tws, stream));
    // one corrected-seminormal-equations step: Z1 = Z0 + R^{-1} R^{-T} (C^T A - C^T C Z0), the
    // products C^T A and C^T C exact with float-float sums, the rest FP64
    SK_CUDA(launch_gemm_tn_ff(m, n, s, static_cast<const float*>(C), m, static_cast<const float*>(A), lda, D, n, fws,
                              "gemm_refine", stream));
    SK_CUDA(launch_gemm_tn_ff(m, s, s, static_cast<const float*>(C), m, static_cast<const float*>(C), m, G, s, fws,
                              "gemm_refine", stream));
    GemmArgs h{};
    h.M = s; h.N = n; h.K = s;
    h.L = View{G, s, 1}; h.l_dt = SKEL_F64;
    h.B = View{Z, ldz, 1}; h.b_dt = SKEL_F64;
    h.out = D; h.out_sr = n; h.out_sc = 1; h.out_dt = SKEL_F64;
    h.alpha = -1.0;
    h.timer = "gemm_refine";
    SK_CUDA(launch_gemm(h, true, LEFT_LOAD, EPI_ACCUM, stream));                    // D = C^T A - C^T C Z0
    SK_CUDA(launch_trsm_upper_t(s, n, R, s, U, D, n, stream));                       // D <- R^{-T} D
    SK_CUDA(launch_trsm_upper(s, n, R, s, 0, SKEL_F64, D, n, D, n, stream));         // D <- R^{-1} D
    SK_CUDA(launch_axpy_rows_f64(s, n, D, n, Z, ldz, stream));                      // Z1 = Z0 + D
    SK_CUDA(launch_unit_columns(s, Js, Z, ldz, stream));
    if (sq_norms) {
      SK_CUDA(launch_sqnorm(m, n, dtype, A, lda, pa, stream));
      SK_CUDA(launch_reduce_sum(pa, nba, sq_norms, 0, stream));
      SK_CUDA(launch_reduce_sum(pw, nbw, sq_norms + 1, 0, stream));
    }
  }
  return SKEL_OK;
}

skel_status skel_pivot_rows(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                            int32_t s, const int32_t* Js, int32_t* Is, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Is == nullptr) return SKEL_ERR_INVALID_ARG;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void* C = ar.take(esize(dtype) * (size_t)m * s);
    const size_t lw = lupp_auto_workspace(dtype, m, s);
    void* lws = ar.take(lw);
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    SK_CUDA(launch_gather_cols(m, s, dtype, A, lda, n, Js, C, m, stream));
    // C column-major m x s is C^T row-major s x m: row pivots of C = column pivots of C^T
    SK_TRY(run_lupp_auto(dtype, C, m, m, s, Is, nullptr, 0, nullptr, 0, lws, lw, dev_status, stream));
  }
  return SKEL_OK;
}

// The stable CUR of Remark 3 (skel_cur), and with `refine` one FP64 refinement step of U.
static skel_status cur_impl(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                            const int32_t* Js, int32_t* Is, int rows_given, double* U, int64_t ldu, double* sq_norms,
                            bool refine, void* ws, size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Is == nullptr || U == nullptr || ldu < s)
    return SKEL_ERR_INVALID_ARG;
  if (refine && dtype != SKEL_F32) return SKEL_ERR_UNSUPPORTED;
  const bool f64 = dtype == SKEL_F64;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void *C, *Qc, *Rt, *Qr;
    double *Rc, *Rr;
    SK_TRY(skeleton_qr(ar, run, m, n, dtype, A, lda, s, Js, &C, &Qc, &Rc, dev_status, stream));
    const size_t lw = rows_given ? 0 : lupp_auto_workspace(dtype, m, s);
    void* lws = rows_given ? nullptr : ar.take(lw);
    Rt = ar.take(esize(dtype) * (size_t)n * s);
    Qr = ar.take(esize(dtype) * (size_t)n * s);
    Rr = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const size_t qn = qr_workspace(dtype, n, s);
    void* qws = ar.take(qn);
    void* W = ar.take(esize(dtype) * (size_t)s * n);
    double* M = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    double* T1 = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    double* T2 = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const int64_t nbm = gemm_num_blocks(s, s);
    double* pm = static_cast<double*>(ar.take(sizeof(double) * nbm));
    const int64_t nba = sqnorm_num_blocks(m, n);
    double* pa = static_cast<double*>(ar.take(sizeof(double) * nba));
    const bool tcw = !f64 && gemm_tc_usable(m, n, s, nullptr, m, A, lda);   // tensor-core W
    void* kws1 = ar.take(tcw ? gemm_tc_workspace(m, n, s) : gemm_workspace(s, n, m, f64));
    void* kws2 = ar.take(gemm_workspace(s, s, n, f64));
    // refinement scratch: C^T A (s x n), C^T C, R R^T, the correction and J R^T J (s x s, FP64)
    double* B1 = refine ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * n)) : nullptr;
    double* Gc = refine ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* Gr = refine ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* D = refine ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* Uf = refine ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    void* fws = refine ? ar.take(std::max({gemm_tn_ff_workspace(m, n, s), gemm_tn_ff_workspace(m, s, s),
                                           gemm_tn_ff_workspace(n, s, s)}))
                       : nullptr;
    void* kws3 = refine ? ar.take(gemm_workspace(s, s, n, true)) : nullptr;
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    // rows by LUPP on C (Algorithm 2, row pivoting): C column-major m x s is C^T row-major s x m
    if (!rows_given)
      SK_TRY(run_lupp_auto(dtype, C, m, m, s, Is, nullptr, 0, nullptr, 0, lws, lw, dev_status, stream));
    SK_CUDA(launch_gather_rows_t(n, s, dtype, A, lda, m, Is, Rt, n, stream));
    SK_TRY(run_qr(dtype, Rt, n, n, s, Qr, n, Rr, s, qws, qn, dev_status, stream));
    GemmArgs g{};
    g.splitk_ws = kws1;
    g.M = s; g.N = n; g.K = m;
    g.L = View{Qc, m, 1}; g.l_dt = dtype;
    g.B = View{A, 1, lda}; g.b_dt = dtype;
    g.out = W; g.out_sr = n; g.out_sc = 1; g.out_dt = dtype;
    g.alpha = 1.0;
    if (tcw)
      SK_CUDA(launch_gemm_tc_tn(m, n, s, static_cast<const float*>(Qc), m, static_cast<const float*>(A), lda,
                                static_cast<float*>(W), n, nullptr, kws1, dev_status, stream));
    else
      SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, stream));
    GemmArgs h{};
    h.splitk_ws = kws2;
    h.M = s; h.N = s; h.K = n;
    h.L = View{W, n, 1}; h.l_dt = dtype;
    h.B = View{Qr, 1, n}; h.b_dt = dtype;
    h.out = M; h.out_sr = s; h.out_sc = 1; h.out_dt = SKEL_F64;
    h.alpha = 1.0;
    h.partials = pm;
    h.timer = "gemm_cur";
    SK_CUDA(launch_gemm(h, f64, LEFT_LOAD, EPI_STORE_SQ, stream));
    if (sq_norms) {
      SK_CUDA(launch_sqnorm(m, n, dtype, A, lda, pa, stream));
      SK_CUDA(launch_reduce_sum(pa, nba, sq_norms, 0, stream));
      SK_CUDA(launch_reduce_sum(pm, nbm, sq_norms + 1, 0, stream));
    }
    // U = R_C^{-1} M R_R^{-T} = (R_R^{-1} (R_C^{-1} M)^T)^T
    SK_CUDA(launch_trsm_upper(s, s, Rc, s, 0, SKEL_F64, M, s, T1, s, stream));
    SK_CUDA(launch_transpose_f64(s, T1, s, T2, s, stream));
    SK_CUDA(launch_trsm_upper(s, s, Rr, s, 0, SKEL_F64, T2, s, T1, s, stream));
    SK_CUDA(launch_transpose_f64(s, T1, s, U, ldu, stream));
    if (!refine) continue;
    // U1 = U0 + (R_C^T R_C)^{-1} (C^T A R^T - (C^T C) U0 (R R^T)) (R_R^T R_R)^{-1}, with C^T A,
    // C^T C and R R^T from exact FP32 products in float-float sums and the rest FP64
    const float* Cf = static_cast<const float*>(C);
    const float* Rf = static_cast<const float*>(Rt);          // R^T, n x s column-major
    SK_CUDA(launch_gemm_tn_ff(m, n, s, Cf, m, static_cast<const float*>(A), lda, B1, n, fws, "gemm_refine", stream));
    SK_CUDA(launch_gemm_tn_ff(m, s, s, Cf, m, Cf, m, Gc, s, fws, "gemm_refine", stream));
    SK_CUDA(launch_gemm_tn_ff(n, s, s, Rf, n, Rf, n, Gr, s, fws, "gemm_refine", stream));
    auto gemm64 = [&](int64_t K, View L, skel_dtype ldt, View B, skel_dtype bdt, double* out, double alpha,
                      GemmEpi epi, void* kws) {
      GemmArgs q{};
      q.splitk_ws = kws;
      q.M = s; q.N = s; q.K = K;
      q.L = L; q.l_dt = ldt;
      q.B = B; q.b_dt = bdt;
      q.out = out; q.out_sr = s; q.out_sc = 1; q.out_dt = SKEL_F64;
      q.alpha = alpha;
      q.timer = "gemm_refine";
      return launch_gemm(q, true, LEFT_LOAD, epi, stream);
    };
    SK_CUDA(gemm64(n, View{B1, n, 1}, SKEL_F64, View{Rf, 1, n}, SKEL_F32, D, 1.0, EPI_STORE, kws3));   // C^T A R^T
    SK_CUDA(gemm64(s, View{Gc, s, 1}, SKEL_F64, View{U, ldu, 1}, SKEL_F64, T1, 1.0, EPI_STORE, nullptr));
    SK_CUDA(gemm64(s, View{T1, s, 1}, SKEL_F64, View{Gr, s, 1}, SKEL_F64, D, -1.0, EPI_ACCUM, nullptr));
    SK_CUDA(launch_trsm_upper_t(s, s, Rc, s, Uf, D, s, stream));                  // R_C^{-T} D
    SK_CUDA(launch_trsm_upper(s, s, Rc, s, 0, SKEL_F64, D, s, D, s, stream));       // R_C^{-1} (.)
    SK_CUDA(launch_transpose_f64(s, D, s, T2, s, stream));                          // E^T
    SK_CUDA(launch_trsm_upper_t(s, s, Rr, s, Uf, T2, s, stream));                 // R_R^{-T} E^T
    SK_CUDA(launch_trsm_upper(s, s, Rr, s, 0, SKEL_F64, T2, s, T2, s, stream));     // R_R^{-1} (.)
    SK_CUDA(launch_transpose_f64(s, T2, s, T1, s, stream));
    SK_CUDA(launch_axpy_rows_f64(s, s, T1, s, U, ldu, stream));                     // U1 = U0 + E (R_R^T R_R)^{-1}
  }
  return SKEL_OK;
}

skel_status skel_cur(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                     int32_t s, const int32_t* Js, int32_t* Is, int rows_given, double* U,
                     int64_t ldu, double* sq_norms, void* ws, size_t* ws_bytes,
                     int32_t* dev_status, cudaStream_t stream) {
  return cur_impl(m, n, dtype, A, lda, s, Js, Is, rows_given, U, ldu, sq_norms, false, ws, ws_bytes, dev_status,
                  stream);
}

skel_status skel_cur_refine(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                            int32_t s, const int32_t* Js, int32_t* Is, int rows_given, double* U,
                            int64_t ldu, double* sq_norms, void* ws, size_t* ws_bytes,
                            int32_t* dev_status, cudaStream_t stream) {
  return cur_impl(m, n, dtype, A, lda, s, Js, Is, rows_given, U, ldu, sq_norms, true, ws, ws_bytes, dev_status,
                  stream);
}

skel_status skel_id_cur(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                        const int32_t* Js, const int32_t* Is, double* Z, int64_t ldz, double* U, int64_t ldu,
                        double* sq_id, double* sq_cur, void* ws, size_t* ws_bytes, int32_t* dev_status,
                        cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Is == nullptr || Z == nullptr || ldz < n || U == nullptr ||
      ldu < s)
    return SKEL_ERR_INVALID_ARG;
  const bool f64 = dtype == SKEL_F64;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    // Two chains.  Caller's stream: QR of C, W = Q_C^T A, Z = R_C^{-1} W, the ID's norms.
    // Auxiliary stream: R^T = A(Is, :)^T and its QR (from the start), then, once W exists,
    // M = W Q_R and U = R_C^{-1} M R_R^{-T}.  The fork comes before the QR of C is enqueued.
    std::unique_lock<std::mutex> lock(aux_mutex(), std::defer_lock);
    AuxSet* aux = nullptr;
    if (run) {
      lock.lock();
      aux = aux_set();
      if (aux == nullptr) return SKEL_ERR_CUDA;
      SK_CUDA(cudaEventRecord(aux->fork, stream));
      SK_CUDA(cudaStreamWaitEvent(aux->st, aux->fork, 0));
    }
    AuxJoin joiner{stream, aux};          // joins on every return path below
    void *C, *Qc;
    double* Rc;
    SK_TRY(skeleton_qr(ar, run, m, n, dtype, A, lda, s, Js, &C, &Qc, &Rc, dev_status, stream));
    void* Rt = ar.take(esize(dtype) * (size_t)n * s);
    void* Qr = ar.take(esize(dtype) * (size_t)n * s);
    double* Rr = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const size_t qn = qr_workspace(dtype, n, s);
    void* qws = ar.take(qn);
    void* W = ar.take(esize(dtype) * (size_t)s * n);
    double* M = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    double* T1 = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    double* T2 = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const bool tcw = !f64 && gemm_tc_usable(m, n, s, nullptr, m, A, lda);   // tensor-core W
    const int64_t nbw = tcw ? gemm_tc_num_partials(m, n, s) : gemm_num_blocks(s, n);
    double* pw = static_cast<double*>(ar.take(sizeof(double) * nbw));
    const int64_t nbm = gemm_num_blocks(s, s);
    double* pm = static_cast<double*>(ar.take(sizeof(double) * nbm));
    const int64_t nba = sqnorm_num_blocks(m, n);
    double* pa = static_cast<double*>(ar.take(sizeof(double) * nba));
    void* kws1 = ar.take(tcw ? gemm_tc_workspace(m, n, s) : gemm_workspace(s, n, m, f64));
    void* kws2 = ar.take(gemm_workspace(s, s, n, f64));
    void* tws = f64 ? nullptr : ar.take(trsm_ff_workspace(s));
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    cudaEvent_t w_ready = aux->col[0];
    // auxiliary chain, part 1: R^T and its QR, concurrent with the QR of C
    SK_CUDA(launch_gather_rows_t(n, s, dtype, A, lda, m, Is, Rt, n, aux->st));
    SK_TRY(run_qr(dtype, Rt, n, n, s, Qr, n, Rr, s, qws, qn, dev_status, aux->st));
    // caller's chain: W = Q_C^T A (with ||W||_F^2), as skel_id
    GemmArgs g{};
    g.splitk_ws = kws1;
    g.M = s; g.N = n; g.K = m;
    g.L = View{Qc, m, 1}; g.l_dt = dtype;
    g.B = View{A, 1, lda}; g.b_dt = dtype;
    g.out = W; g.out_sr = n; g.out_sc = 1; g.out_dt = dtype;
    g.alpha = 1.0;
    g.partials = pw;
    if (tcw)
      SK_CUDA(launch_gemm_tc_tn(m, n, s, static_cast<const float*>(Qc), m, static_cast<const float*>(A), lda,
                                static_cast<float*>(W), n, pw, kws1, dev_status, stream));
    else
      SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_STORE_SQ, stream));
    SK_CUDA(cudaEventRecord(w_ready, stream));
    // auxiliary chain, part 2: M = W Q_R = Q_C^T A Q_R and U = R_C^{-1} M R_R^{-T}, as skel_cur,
    // concurrent with the solve for Z
    SK_CUDA(cudaStreamWaitEvent(aux->st, w_ready, 0));
    GemmArgs h{};
    h.splitk_ws = kws2;
    h.M = s; h.N = s; h.K = n;
    h.L = View{W, n, 1}; h.l_dt = dtype;
    h.B = View{Qr, 1, n}; h.b_dt = dtype;
    h.out = M; h.out_sr = s; h.out_sc = 1; h.out_dt = SKEL_F64;
    h.alpha = 1.0;
    h.partials = pm;
    h.timer = "gemm_cur";
    SK_CUDA(launch_gemm(h, f64, LEFT_LOAD, EPI_STORE_SQ, aux->st));
    SK_CUDA(launch_trsm_upper(s, s, Rc, s, 0, SKEL_F64, M, s, T1, s, aux->st));
    SK_CUDA(launch_transpose_f64(s, T1, s, T2, s, aux->st));
    SK_CUDA(launch_trsm_upper(s, s, Rr, s, 0, SKEL_F64, T2, s, T1, s, aux->st));
    SK_CUDA(launch_transpose_f64(s, T1, s, U, ldu, aux->st));
    // caller's chain: Z = R_C^{-1} W and the norms
    if (f64)
      SK_CUDA(launch_trsm_upper(s, n, Rc, s, 0, dtype, W, n, Z, ldz, stream));
    else    // the FP32 W in float-float arithmetic (FP32 pipes)
      SK_CUDA(launch_trsm_upper_ff(s, n, Rc, s, static_cast<const float*>(W), n, Z, ldz, tws, stream));
    if (sq_id || sq_cur) SK_CUDA(launch_sqnorm(m, n, dtype, A, lda, pa, stream));
    if (sq_id) {
      SK_CUDA(launch_reduce_sum(pa, nba, sq_id, 0, stream));
      SK_CUDA(launch_reduce_sum(pw, nbw, sq_id + 1, 0, stream));
    }
    SK_CUDA(cudaEventRecord(aux->join, aux->st));
    SK_CUDA(cudaStreamWaitEvent(stream, aux->join, 0));
    if (sq_cur) {
      SK_CUDA(launch_reduce_sum(pa, nba, sq_cur, 0, stream));
      SK_CUDA(launch_reduce_sum(pm, nbm, sq_cur + 1, 0, stream));
    }
  }
  return SKEL_OK;
}

skel_status skel_cur_sketch(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda, int32_t s,
                            const int32_t* Js, const int32_t* Is, double* U, int64_t ldu, void* ws,
                            size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (!id_args_ok(m, n, dtype, A, lda, s, Js) || Is == nullptr || U == nullptr || ldu < s) return SKEL_ERR_INVALID_ARG;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void* C = ar.take(esize(dtype) * (size_t)m * s);
    void* St = ar.take(esize(dtype) * (size_t)s * s);          // S^T, column-major
    void* Q = ar.take(esize(dtype) * (size_t)s * s);
    double* R = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    double* V = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const size_t qn = qr_workspace(dtype, s, s);
    void* qws = ar.take(qn);
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    SK_CUDA(launch_gather_cols(m, s, dtype, A, lda, n, Js, C, m, stream));           // C = A(:, J)
    SK_CUDA(launch_gather_rows_t(s, s, dtype, C, m, m, Is, St, s, stream));          // S^T(c, r) = C(I_r, c)
    SK_TRY(run_qr(dtype, St, s, s, s, Q, s, R, s, qws, qn, dev_status, stream));   // S^T = Q R
    SK_CUDA(launch_trsm_upper(s, s, R, s, 0, dtype, Q, s, V, s, stream));          // V = R^{-1} Q^T
    SK_CUDA(launch_transpose_f64(s, V, s, U, ldu, stream));                       // U = V^T = S^{-1}
  }
  return SKEL_OK;
}

skel_status skel_id_sketch(skel_dtype dtype, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                           const int32_t* Js, double* Z, int64_t ldz, void* ws, size_t* ws_bytes,
                           int32_t* dev_status, cudaStream_t stream) {
  if (!valid_dtype(dtype) || X == nullptr || Js == nullptr || Z == nullptr || s < 1 || s > kMaxS || l < s ||
      l > 4096 || n < s || n > (int64_t)INT32_MAX || ldx < n || ldz < n)
    return SKEL_ERR_INVALID_ARG;
  const bool f64 = dtype == SKEL_F64;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    void* X1 = ar.take(esize(dtype) * (size_t)l * s);
    void* Q = ar.take(esize(dtype) * (size_t)l * s);
    double* R1 = static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s));
    const size_t qn = qr_workspace(dtype, l, s);
    void* qws = ar.take(qn);
    void* W = ar.take(esize(dtype) * (size_t)s * n);
    void* kws = ar.take(gemm_workspace(s, n, l, f64));
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    // X1 = X(:, J) as an l x s column-major matrix: the row gather of X^T (n x l column-major)
    SK_CUDA(launch_gather_rows_t(l, s, dtype, X, ldx, n, Js, X1, l, stream));
    SK_TRY(run_qr(dtype, X1, l, l, s, Q, l, R1, s, qws, qn, dev_status, stream));     // X1 = Q R1
    GemmArgs g{};
    g.splitk_ws = kws;
    g.M = s; g.N = n; g.K = l;
    g.L = View{Q, l, 1}; g.l_dt = dtype;          // Q^T(t, r) = Q(r, t)
    g.B = View{X, ldx, 1}; g.b_dt = dtype;        // X(r, j), row-major
    g.out = W; g.out_sr = n; g.out_sc = 1; g.out_dt = dtype;
    g.alpha = 1.0;
    g.dev_status = dev_status;
    SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, stream));                        // W = Q^T X
    SK_CUDA(launch_trsm_upper(s, n, R1, s, 0, dtype, W, n, Z, ldz, stream));           // Z = R1^{-1} W
    SK_CUDA(launch_unit_columns(s, Js, Z, ldz, stream));                               // Z(:, J) = I exactly
  }
  return SKEL_OK;
}

skel_status skel_error(int64_t m, int64_t n, skel_dtype dtype, const void* A, int64_t lda,
                       int32_t s, const int32_t* Js, const double* Z, int64_t ldz,
                       const int32_t* Is, const double* U, int64_t ldu, skel_dtype rf_dtype,
                       const void* Rf, int64_t ldrf, double* out, void* ws, size_t* ws_bytes,
                       int32_t* dev_status, cudaStream_t stream) {
  if (!valid_dtype(dtype) || A == nullptr || out == nullptr || m < 1 || n < 1 || lda < m)
    return SKEL_ERR_INVALID_ARG;
  const bool need_js = Z || U || Rf;
  if (need_js && (Js == nullptr || s < 1 || s > kMaxS || s > m || s > n)) return SKEL_ERR_INVALID_ARG;
  if ((Z && ldz < n) || (U && (ldu < s || Is == nullptr)) || (Rf && (!valid_dtype(rf_dtype) || ldrf < n)))
    return SKEL_ERR_INVALID_ARG;
  const bool f64 = dtype == SKEL_F64;
  for (int pass = 0; pass < 2; ++pass) {
    const bool run = pass == 1;
    Arena ar(run ? ws : nullptr);
    const int64_t nba = sqnorm_num_blocks(m, n);
    double* pa = static_cast<double*>(ar.take(sizeof(double) * nba));
    void* C = need_js ? ar.take(esize(dtype) * (size_t)m * s) : nullptr;
    const int64_t nbr = gemm_num_blocks(m, n);
    double* pr = static_cast<double*>(ar.take(sizeof(double) * nbr));
    void* P = U ? ar.take(esize(dtype) * (size_t)m * s) : nullptr;
    void* Rt = U ? ar.take(esize(dtype) * (size_t)n * s) : nullptr;
    double* H = Rf ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* R1 = Rf ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* M1 = Rf ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* M2 = Rf ? static_cast<double*>(ar.take(sizeof(double) * (size_t)s * s)) : nullptr;
    double* pscr = Rf ? static_cast<double*>(ar.take(power_scratch_bytes(s))) : nullptr;
    const bool ffh = Rf && rf_dtype == SKEL_F32;     // FP32 R: float-float R R^T
    void* kwsh = Rf ? ar.take(ffh ? syrk_ff_workspace(s, n) : gemm_workspace(s, s, n, true)) : nullptr;
    if (!run) {
      skel_status st;
      if (ws_handshake(ar.off, ws, ws_bytes, &st)) return st;
      continue;
    }
    SK_CUDA(launch_fill_f64(out, 4, NAN, stream));
    SK_CUDA(launch_sqnorm(m, n, dtype, A, lda, pa, stream));
    SK_CUDA(launch_reduce_sum(pa, nba, out + 0, 1, stream));
    if (need_js) SK_CUDA(launch_gather_cols(m, s, dtype, A, lda, n, Js, C, m, stream));
    if (Z) {
      GemmArgs g{};
      g.M = m; g.N = n; g.K = s;
      g.L = View{C, 1, m}; g.l_dt = dtype;
      g.B = View{Z, ldz, 1}; g.b_dt = SKEL_F64;
      g.ref = View{A, 1, lda}; g.ref_dt = dtype;
      g.alpha = 1.0;
      g.partials = pr;
      SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_RESID, stream));
      SK_CUDA(launch_reduce_sum(pr, nbr, out + 1, 1, stream));
    }
    if (U) {
      GemmArgs g{};
      g.M = m; g.N = s; g.K = s;
      g.L = View{C, 1, m}; g.l_dt = dtype;
      g.B = View{U, ldu, 1}; g.b_dt = SKEL_F64;
      g.out = P; g.out_sr = 1; g.out_sc = m; g.out_dt = dtype;
      g.alpha = 1.0;
      SK_CUDA(launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, stream));
      SK_CUDA(launch_gather_rows_t(n, s, dtype, A, lda, m, Is, Rt, n, stream));
      GemmArgs h{};
      h.M = m; h.N = n; h.K = s;
      h.L = View{P, 1, m}; h.l_dt = dtype;
      h.B = View{Rt, n, 1}; h.b_dt = dtype;          // R(r, c) = Rt[c + r*n]
      h.ref = View{A, 1, lda}; h.ref_dt = dtype;
      h.alpha = 1.0;
      h.partials = pr;
      SK_CUDA(launch_gemm(h, f64, LEFT_LOAD, EPI_RESID, stream));
      SK_CUDA(launch_reduce_sum(pr, nbr, out + 2, 1, stream));
    }
    if (Rf) {
      // eta^2 = lambda_max(R_1^{-1} (R R^T) R_1^{-T}) = 1 + ||R_1^{-1} R_2||_2^2
      GemmArgs g{};
      g.splitk_ws = kwsh;
      g.M = s; g.N = s; g.K = n;
      g.L = View{Rf, ldrf, 1}; g.l_dt = rf_dtype;
      g.B = View{Rf, 1, ldrf}; g.b_dt = rf_dtype;
      g.out = H; g.out_sr = s; g.out_sc = 1; g.out_dt = SKEL_F64;
      g.alpha = 1.0;
      g.timer = "gemm_eta_h";
      if (ffh)
        SK_CUDA(launch_syrk_ff(s, n, static_cast<const float*>(Rf), ldrf, H, s, kwsh, stream));
      else
        SK_CUDA(launch_gemm(g, true, LEFT_LOAD, EPI_STORE, stream));
      SK_CUDA(launch_gather_cols_rowmajor_f64(s, rf_dtype, Rf, ldrf, n, Js, R1, s, stream));
      SK_CUDA(launch_trsm_upper(s, s, R1, s, 0, SKEL_F64, H, s, M1, s, stream));
      SK_CUDA(launch_transpose_f64(s, M1, s, M2, s, stream));
      SK_CUDA(launch_trsm_upper(s, s, R1, s, 0, SKEL_F64, M2, s, M1, s, stream));
      SK_CUDA(launch_power_sqrt_lmax(s, M1, s, out + 3, pscr, stream));
    }
  }
  return SKEL_OK;
}

}  // extern "C"
