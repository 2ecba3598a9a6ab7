// Householder QR of the tall skeleton C = A(:, Js) (m x s), for the column ID
// Z = R_C^{-1} Q_C^T A (Eq. (2.1)) and the stable CUR of Remark 3 (also applied to R^T).
//
// One persistent cooperative grid; CTA b owns a contiguous block of rows, resident in shared
// memory (global workspace when too large).  Step t of the factorization needs the dot
// products of column t with columns t..s-1 over rows >= t (a "Gram row"); then
//     beta = -sign(alpha) ||x||,  v = (x - beta e_t)/(alpha - beta),  tau = (beta - alpha)/beta,
//     v^T C(:, j) = (D_j - beta C(t, j)) / (alpha - beta),
// and every CTA updates its rows; R(t, :) = C(t, :) - tau v^T C(:, :) is known everywhere.
// The Gram row is reduced in two barriers: (A) every CTA publishes its partial row (and the
// owner of row t publishes row t); (B) CTA b sums the G partials of columns t+b, t+b+G, ...
// in a fixed order and writes them, with row t, to a reduced buffer; every CTA then reads
// the s-t reduced values.  The explicit Q_C = H_0 ... H_{s-1} [I_s; 0] is accumulated
// backwards with the same two-barrier reduction per reflector.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 200 * 1024;

template <typename T>
struct QrParams {
  const T* C; int64_t m, ldc; int s;
  T* Q; int64_t ldq;
  double* R; int64_t ldr;
  T* gblock;          // global storage for [B | Y] when not in shared memory
  T* red;             // reduced buffers [2][2s]
  int mloc, in_smem;
  GridComm gc;
  int32_t* dev_status;
};

__device__ __forceinline__ unsigned char* carve(unsigned char*& p, size_t bytes) {
  unsigned char* r = p;
  p += (bytes + 15) & ~size_t(15);
  return r;
}

// Phase B of a two-barrier reduction for Gram-row step `k` (barrier indices 2k, 2k+1):
// this CTA reduces its share of columns [lo, s) and, when `with_row`, copies row values
// [lo, s) from the owner's slot.  Then arrive + wait, and every CTA reads the result into
// red_s[lo..s) (and row_s).
template <typename T>
__device__ __forceinline__ bool reduce_gram(const QrParams<T>& p, int k, int lo, bool with_row, int owner,
                                            T* red_s, T* row_s) {
  const int G = p.gc.G, s = p.s, b = blockIdx.x;
  T* out = p.red + (int64_t)(k & 1) * 2 * s;
  for (int j = lo + b + G * (int)threadIdx.x; j < s; j += G * blockDim.x) {
    T acc = T(0);
    for (int q = 0; q < G; ++q) acc += __ldcg(reinterpret_cast<const T*>(p.gc.slot(2 * k, q)) + j);
    out[j] = acc;
    if (with_row) out[s + j] = __ldcg(reinterpret_cast<const T*>(p.gc.slot(2 * k, owner)) + s + j);
  }
  comm_arrive(p.gc, 2 * k + 1);
  if (!comm_wait(p.gc, 2 * k + 1, p.dev_status)) return false;
  for (int j = lo + threadIdx.x; j < s; j += blockDim.x) {
    red_s[j] = __ldcg(out + j);
    if (with_row) row_s[j] = __ldcg(out + s + j);
  }
  __syncthreads();
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) qr_kernel(const QrParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
  const int s = p.s, mloc = p.mloc;
  const int64_t r0 = (int64_t)b * mloc;
  const int ml = (int)(p.m - r0 < 0 ? 0 : (p.m - r0 < mloc ? p.m - r0 : mloc));
  unsigned char* cur = smem;
  T* tau = (T*)carve(cur, sizeof(T) * s);
  T* red = (T*)carve(cur, sizeof(T) * s);     // reduced Gram row / w
  T* rowt = (T*)carve(cur, sizeof(T) * s);    // row t of C at step t
  T* Bm;
  T* Y;
  if (p.in_smem) {
    Bm = (T*)carve(cur, sizeof(T) * (size_t)mloc * s);
    Y = (T*)carve(cur, sizeof(T) * (size_t)mloc * s);
  } else {
    Bm = p.gblock + (int64_t)b * 2 * mloc * s;
    Y = Bm + (int64_t)mloc * s;
  }
  auto B = [&](int i, int j) -> T& { return Bm[(int64_t)j * mloc + i]; };
  auto Yv = [&](int i, int j) -> T& { return Y[(int64_t)j * mloc + i]; };

  for (int64_t e = tid; e < (int64_t)ml * s; e += bd) {
    const int i = (int)(e % ml), j = (int)(e / ml);
    B(i, j) = p.C[r0 + i + (int64_t)j * p.ldc];
  }
  __syncthreads();

  // ---------------- factorization ----------------
  for (int t = 0; t < s; ++t) {
    T* part = reinterpret_cast<T*>(p.gc.slot(2 * t, b));
    T* prow = part + s;
    const int ilo = (int)(t - r0 > 0 ? t - r0 : 0);       // first local row with global index >= t
    for (int j = t + warp; j < s; j += nwarps) {
      T d = T(0);
      for (int i = ilo + lane; i < ml; i += 32) d += B(i, t) * B(i, j);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) part[j] = d;
    }
    const bool owner = (t >= r0 && t < r0 + ml);
    if (owner)
      for (int j = t + tid; j < s; j += bd) prow[j] = B((int)(t - r0), j);
    comm_arrive(p.gc, 2 * t);
    if (!comm_wait(p.gc, 2 * t, p.dev_status)) return;
    if (!reduce_gram(p, t, t, true, t / mloc, red, rowt)) return;
    const T sig2 = red[t];
    const T alpha = rowt[t];
    if (!isfinite(sig2)) {
      if (tid == 0) { record_error(p.dev_status, SKEL_ERR_NONFINITE, t); atomicExch(p.gc.abort, 1); }
      return;
    }
    if (sig2 == T(0)) {
      if (tid == 0) { record_error(p.dev_status, SKEL_ERR_RANK_DEFICIENT, t); atomicExch(p.gc.abort, 1); }
      return;
    }
    const T nrm = sqrt(sig2);
    const T beta = alpha != T(0) ? -copysign(nrm, alpha) : -nrm;
    const T den = alpha - beta;
    const T tt = (beta - alpha) / beta;
    if (tid == 0) tau[t] = tt;
    __syncthreads();
    for (int j = t + 1 + tid; j < s; j += bd) red[j] = (red[j] - beta * rowt[j]) / den;
    __syncthreads();
    if (b == 0) {
      for (int j = tid; j < s; j += bd) {
        double rv;
        if (j < t) rv = 0.0;
        else if (j == t) rv = (double)beta;
        else rv = (double)(rowt[j] - tt * red[j]);
        p.R[(int64_t)t * p.ldr + j] = rv;
      }
    }
    for (int i = ilo + tid; i < ml; i += bd) {
      const int64_t gi = r0 + i;
      if (gi > t) B(i, t) = B(i, t) / den;
    }
    __syncthreads();
    const int ncol = s - t - 1;
    for (int64_t e = tid; e < (int64_t)(ml - ilo) * ncol; e += bd) {
      const int i = ilo + (int)(e % (ml - ilo)), j = t + 1 + (int)(e / (ml - ilo));
      const int64_t gi = r0 + i;
      const T vi = (gi == t) ? T(1) : B(i, t);
      B(i, j) -= tt * vi * red[j];
    }
    __syncthreads();
  }

  // ---------------- Q = H_0 ... H_{s-1} [I; 0], backwards ----------------
  for (int64_t e = tid; e < (int64_t)ml * s; e += bd) {
    const int i = (int)(e % ml), j = (int)(e / ml);
    Yv(i, j) = (r0 + i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    const int u = s - 1 - k;
    const int step = s + k;
    T* part = reinterpret_cast<T*>(p.gc.slot(2 * step, b));
    const int ilo = (int)(u - r0 > 0 ? u - r0 : 0);
    for (int j = u + warp; j < s; j += nwarps) {
      T d = T(0);
      for (int i = ilo + lane; i < ml; i += 32) {
        const T vi = (r0 + i == u) ? T(1) : B(i, u);
        d += vi * Yv(i, j);
      }
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) part[j] = d;
    }
    comm_arrive(p.gc, 2 * step);
    if (!comm_wait(p.gc, 2 * step, p.dev_status)) return;
    if (!reduce_gram(p, step, u, false, 0, red, rowt)) return;
    const T tu = tau[u];
    const int ncol = s - u;
    for (int64_t e = tid; e < (int64_t)(ml - ilo) * ncol; e += bd) {
      const int i = ilo + (int)(e % (ml - ilo)), j = u + (int)(e / (ml - ilo));
      const T vi = (r0 + i == u) ? T(1) : B(i, u);
      Yv(i, j) -= tu * vi * red[j];
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)ml * s; e += bd) {
    const int i = (int)(e % ml), j = (int)(e / ml);
    p.Q[r0 + i + (int64_t)j * p.ldq] = Yv(i, j);
  }
}

struct QrPlan {
  int G, mloc, in_smem, nsteps;
  size_t smem, slot_bytes, comm_bytes, red_bytes, block_bytes, total;
};

template <typename T>
QrPlan plan_qr(int64_t m, int s) {
  QrPlan pl{};
  const int sms = device_sm_count();
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>({(m + 63) / 64, (int64_t)sms, (int64_t)kThreads}));
  pl.mloc = (int)((m + pl.G - 1) / pl.G);
  pl.nsteps = 4 * s;
  auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  const size_t base = 3 * a16(sizeof(T) * s);
  const size_t slab = 2 * a16(sizeof(T) * (size_t)pl.mloc * s);
  pl.in_smem = base + slab <= kSmemBudget;
  pl.smem = pl.in_smem ? base + slab : base;
  pl.slot_bytes = align_up(2 * sizeof(T) * s, 16);
  pl.comm_bytes = comm_header_bytes(1) + align_up(2 * pl.G * pl.slot_bytes);
  pl.red_bytes = align_up(sizeof(T) * 4 * (size_t)s);
  pl.block_bytes = pl.in_smem ? 0 : align_up(sizeof(T) * (size_t)pl.G * 2 * pl.mloc * s);
  pl.total = pl.comm_bytes + pl.red_bytes + pl.block_bytes;
  return pl;
}

template <typename T>
skel_status launch_qr_t(const T* C, int64_t m, int64_t ldc, int s, T* Q, int64_t ldq, double* R,
                        int64_t ldr, void* ws, size_t ws_bytes, int32_t* dev_status,
                        cudaStream_t st) {
  const QrPlan pl = plan_qr<T>(m, s);
  if (ws_bytes < pl.total) return SKEL_ERR_WORKSPACE;
  char* base = static_cast<char*>(ws);
  QrParams<T> p{};
  p.C = C; p.m = m; p.ldc = ldc; p.s = s; p.Q = Q; p.ldq = ldq; p.R = R; p.ldr = ldr;
  p.gc.counter = reinterpret_cast<unsigned int*>(base);
  p.gc.abort = reinterpret_cast<int32_t*>(base + 4);
  p.gc.keys = nullptr;
  p.gc.payload = base + comm_header_bytes(1);
  p.gc.slot_bytes = (int64_t)pl.slot_bytes;
  p.gc.G = pl.G;
  p.gc.wait_ns = kDefaultWaitNs;
  p.red = reinterpret_cast<T*>(base + pl.comm_bytes);
  p.gblock = pl.in_smem ? nullptr : reinterpret_cast<T*>(base + pl.comm_bytes + pl.red_bytes);
  p.mloc = pl.mloc;
  p.in_smem = pl.in_smem;
  p.dev_status = dev_status;
  if (cudaMemsetAsync(base, 0, comm_header_bytes(1), st) != cudaSuccess) return SKEL_ERR_CUDA;
  if (cudaFuncSetAttribute((const void*)qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pl.smem) != cudaSuccess)
    return SKEL_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launches(1);
  return cudaLaunchKernelEx(&cfg, qr_kernel<T>, p) == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

size_t qr_workspace(skel_dtype dt, int64_t m, int32_t s) {
  return dt == SKEL_F64 ? plan_qr<double>(m, s).total : plan_qr<float>(m, s).total;
}

skel_status run_qr(skel_dtype dt, const void* C, int64_t m, int64_t ldc, int32_t s, void* Q,
                   int64_t ldq, double* R, int64_t ldr, void* ws, size_t ws_bytes,
                   int32_t* dev_status, cudaStream_t st) {
  if (dt == SKEL_F64)
    return launch_qr_t<double>((const double*)C, m, ldc, s, (double*)Q, ldq, R, ldr, ws, ws_bytes,
                               dev_status, st);
  return launch_qr_t<float>((const float*)C, m, ldc, s, (float*)Q, ldq, R, ldr, ws, ws_bytes,
                            dev_status, st);
}

}  // namespace skel
