// Householder QR of the tall skeleton C = A(:, Js) (m x s), for the column ID
// Z = R_C^{-1} Q_C^T A (Eq. (2.1)) and the stable CUR of Remark 3 (also applied to R^T).
//
// Factorisation: panels of columns on thread-block clusters (qr_panel.cu) when a panel of at
// least 8 columns fits the cluster's shared memory; otherwise the kernel below.
// Fallback factorisation: one persistent cooperative grid; CTA b owns a contiguous block of rows,
// resident in shared memory (global workspace when too large).  Step t needs the dot
// products of column t with columns t..s-1 over rows >= t (a "Gram row"): every CTA adds its
// partial Gram row into a per-step accumulator with atomics, the owner of row t publishes
// row t, and after one grid barrier every CTA forms
//     beta = -sign(alpha) ||x||,  v = (x - beta e_t)/(alpha - beta),  tau = (beta - alpha)/beta,
//     v^T C(:, j) = (D_j - beta C(t, j)) / (alpha - beta),
// updates its rows, and keeps v in place.  R(t, :) = C(t, :) - tau (v^T C)(:) is known to
// every CTA.  (The accumulation order of the atomics is not fixed, so results can differ
// between runs in the last bits.)
//
// Explicit Q_C: with V = [v_0 .. v_{s-1}] (unit lower trapezoidal) and tau_i = 2/||v_i||^2,
// Q = H_0 ... H_{s-1} = I - V T V^T where T^{-1} = diag(V^T V)/2 + strictly_upper(V^T V)
// (the compact WY representation).  Hence Q_C = Q(:, 0:s) = [I_s; 0] - V (T V_1^T),
// V_1 = V(0:s, :):  G = V^T V (GEMM), S = T^{-1} from G, M = S^{-1} V_1^T (FP64 triangular
// solve), Q_C = -V M + [I_s; 0] (GEMM plus the identity).
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
  T* V; int64_t ldv;           // out: reflectors, unit lower trapezoidal, m x s col-major
  double* R; int64_t ldr;      // out: s x s upper triangular, row-major
  T* acc;                      // [s][s] Gram-row accumulators (zeroed by the host)
  T* rows;                     // [s][s] published rows t
  T* gblock;                   // global slab when not in shared memory
  int mloc, in_smem;
  GridComm gc;
  int32_t* dev_status;
};

__device__ __forceinline__ unsigned char* carve(unsigned char*& p, size_t bytes) {
  unsigned char* r = p;
  p += (bytes + 15) & ~size_t(15);
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) qr_factor_kernel(const QrParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
  const int s = p.s, mloc = p.mloc;
  const int64_t r0 = (int64_t)b * mloc;
  const int ml = (int)(p.m - r0 < 0 ? 0 : (p.m - r0 < mloc ? p.m - r0 : mloc));
  unsigned char* cur = smem;
  T* red = (T*)carve(cur, sizeof(T) * s);     // reduced Gram row, then w
  T* rowt = (T*)carve(cur, sizeof(T) * s);    // row t of C at step t
  T* Bm = p.in_smem ? (T*)carve(cur, sizeof(T) * (size_t)mloc * s) : p.gblock + (int64_t)b * mloc * s;
  auto B = [&](int i, int j) -> T& { return Bm[(int64_t)j * mloc + i]; };

  for (int j = 0; j < s; ++j)
    for (int i = tid; i < ml; i += bd) B(i, j) = p.C[r0 + i + (int64_t)j * p.ldc];
  __syncthreads();

  for (int t = 0; t < s; ++t) {
    const int ilo = (int)(t - r0 > 0 ? t - r0 : 0);       // first local row with global index >= t
    T* acc = p.acc + (int64_t)t * s;
    if (ilo < ml) {
      for (int j = t + warp; j < s; j += nwarps) {
        T d = T(0);
        for (int i = ilo + lane; i < ml; i += 32) d += B(i, t) * B(i, j);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) atomicAdd(acc + j, d);
      }
    }
    if (t >= r0 && t < r0 + ml)
      for (int j = t + tid; j < s; j += bd) p.rows[(int64_t)t * s + j] = B((int)(t - r0), j);
    comm_arrive(p.gc, t);
    if (!comm_wait(p.gc, t, p.dev_status)) return;
    for (int j = t + tid; j < s; j += bd) {
      red[j] = __ldcg(acc + j);
      rowt[j] = __ldcg(p.rows + (int64_t)t * s + j);
    }
    __syncthreads();
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
    // rows over lanes, columns over warps: no integer division in the loop
    for (int j = t + 1 + warp; j < s; j += nwarps) {
      const T f = tt * red[j];
      for (int i = ilo + lane; i < ml; i += 32) {
        const T vi = (r0 + i == t) ? T(1) : B(i, t);
        B(i, j) -= f * vi;
      }
    }
    __syncthreads();
  }
  // V: explicit unit diagonal and zeros above it
  for (int j = 0; j < s; ++j)
    for (int i = tid; i < ml; i += bd) {
      const int64_t gi = r0 + i;
      p.V[gi + (int64_t)j * p.ldv] = gi > j ? B(i, j) : (gi == j ? T(1) : T(0));
    }
}

// S = diag(G)/2 + strictly_upper(G) (= T^{-1} of the compact WY form), s x s row-major FP64.
__global__ void wy_tinv_kernel(int s, const double* G, double* S) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / s), j = (int)(e % s);
    S[e] = j > i ? G[e] : (j == i ? 0.5 * G[e] : 0.0);
  }
}

template <typename T>
__global__ void add_identity_kernel(int s, T* Q, int64_t ldq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) Q[i + (int64_t)i * ldq] += T(1);
}

struct QrPlan {
  int G, mloc, in_smem;
  size_t smem, comm_bytes, acc_bytes, block_bytes, factor_total;
};

template <typename T>
QrPlan plan_qr(int64_t m, int s) {
  QrPlan pl{};
  const int sms = device_sm_count();
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>({(m + 63) / 64, (int64_t)sms, (int64_t)kThreads}));
  pl.mloc = (int)((m + pl.G - 1) / pl.G);
  auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  const size_t base = 2 * a16(sizeof(T) * s);
  const size_t slab = a16(sizeof(T) * (size_t)pl.mloc * s);
  pl.in_smem = base + slab <= kSmemBudget;
  pl.smem = pl.in_smem ? base + slab : base;
  pl.comm_bytes = comm_header_bytes(1);
  pl.acc_bytes = align_up(sizeof(T) * (size_t)s * s);
  pl.block_bytes = pl.in_smem ? 0 : align_up(sizeof(T) * (size_t)pl.G * pl.mloc * s);
  pl.factor_total = pl.comm_bytes + 2 * pl.acc_bytes + pl.block_bytes;
  return pl;
}

// Workspace of the Q formation after the factorisation: V (m x s), G, S, M (s x s FP64),
// split-K scratch for G = V^T V and for Q = -V M.
template <typename T>
size_t q_extra_bytes(int64_t m, int s) {
  const bool f64 = sizeof(T) == 8;
  return align_up(sizeof(T) * (size_t)m * s) + 3 * align_up(sizeof(double) * (size_t)s * s) +
         gemm_workspace(s, s, m, f64) + gemm_workspace(m, s, s, f64);
}

template <typename T>
skel_status launch_qr_t(const T* C, int64_t m, int64_t ldc, int s, T* Q, int64_t ldq, double* R,
                        int64_t ldr, void* ws, size_t ws_bytes, int32_t* dev_status,
                        cudaStream_t st) {
  const QrPlan pl = plan_qr<T>(m, s);
  const bool f64 = sizeof(T) == 8;
  const skel_dtype dt = f64 ? SKEL_F64 : SKEL_F32;
  const size_t pws = qr_panels_workspace(dt, m, s);     // 0: panels do not fit a cluster
  const size_t factor = pws > 0 ? pws : pl.factor_total;
  if (ws_bytes < factor + q_extra_bytes<T>(m, s)) return SKEL_ERR_WORKSPACE;
  char* base = static_cast<char*>(ws);
  QrParams<T> p{};
  p.C = C; p.m = m; p.ldc = ldc; p.s = s; p.R = R; p.ldr = ldr;
  p.gc.counter = reinterpret_cast<unsigned int*>(base);
  p.gc.abort = reinterpret_cast<int32_t*>(base + 4);
  p.gc.keys = nullptr;
  p.gc.payload = nullptr;
  p.gc.slot_bytes = 0;
  p.gc.G = pl.G;
  p.gc.wait_ns = kDefaultWaitNs;
  p.acc = reinterpret_cast<T*>(base + pl.comm_bytes);
  p.rows = reinterpret_cast<T*>(base + pl.comm_bytes + pl.acc_bytes);
  p.gblock = pl.in_smem ? nullptr : reinterpret_cast<T*>(base + pl.comm_bytes + 2 * pl.acc_bytes);
  p.mloc = pl.mloc;
  p.in_smem = pl.in_smem;
  p.dev_status = dev_status;
  char* extra = base + factor;
  T* V = reinterpret_cast<T*>(extra);
  extra += align_up(sizeof(T) * (size_t)m * s);
  double* Gm = reinterpret_cast<double*>(extra);
  extra += align_up(sizeof(double) * (size_t)s * s);
  double* Sm = reinterpret_cast<double*>(extra);
  extra += align_up(sizeof(double) * (size_t)s * s);
  double* Mm = reinterpret_cast<double*>(extra);
  extra += align_up(sizeof(double) * (size_t)s * s);
  void* kws1 = extra;
  extra += gemm_workspace(s, s, m, f64);
  void* kws2 = extra;
  p.V = V; p.ldv = m;

  if (pws > 0)        // factorisation and Q_C from the panels' WY blocks
    return run_qr_panels(dt, C, m, ldc, s, V, m, R, ldr, Q, ldq, base, pws, dev_status, st);
  {
  if (cudaMemsetAsync(base, 0, pl.comm_bytes + pl.acc_bytes, st) != cudaSuccess) return SKEL_ERR_CUDA;
  if (cudaFuncSetAttribute((const void*)qr_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  if (cudaLaunchKernelEx(&cfg, qr_factor_kernel<T>, p) != cudaSuccess) return SKEL_ERR_CUDA;
  }

  // G = V^T V (s x s, FP64 out)
  GemmArgs g{};
  g.M = s; g.N = s; g.K = m;
  g.L = View{V, m, 1}; g.l_dt = dt;            // V^T(r, i) = V(i, r)
  g.B = View{V, 1, m}; g.b_dt = dt;
  g.out = Gm; g.out_sr = s; g.out_sc = 1; g.out_dt = SKEL_F64;
  g.alpha = 1.0;
  g.splitk_ws = kws1;
  if (launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, st) != cudaSuccess) return SKEL_ERR_CUDA;
  wy_tinv_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * s + 255) / 256, 1024), 256, 0, st>>>(s, Gm, Sm);
  note_launches(1);
  // M = S^{-1} V_1^T: row i of V_1^T is column i of V (rows 0..s-1), contiguous with stride m
  if (launch_trsm_upper(s, s, Sm, s, 0, dt, V, m, Mm, s, st) != cudaSuccess) return SKEL_ERR_CUDA;
  // Q_C = -V M + [I; 0]
  GemmArgs q{};
  q.M = m; q.N = s; q.K = s;
  q.L = View{V, 1, m}; q.l_dt = dt;
  q.B = View{Mm, s, 1}; q.b_dt = SKEL_F64;
  q.out = Q; q.out_sr = 1; q.out_sc = ldq; q.out_dt = dt;
  q.alpha = -1.0;
  q.splitk_ws = kws2;
  if (launch_gemm(q, f64, LEFT_LOAD, EPI_STORE, st) != cudaSuccess) return SKEL_ERR_CUDA;
  add_identity_kernel<T><<<(s + 255) / 256, 256, 0, st>>>(s, Q, ldq);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

size_t qr_workspace(skel_dtype dt, int64_t m, int32_t s) {
  const size_t pws = qr_panels_workspace(dt, m, s);
  if (dt == SKEL_F64) return (pws > 0 ? pws : plan_qr<double>(m, s).factor_total) + q_extra_bytes<double>(m, s);
  return (pws > 0 ? pws : plan_qr<float>(m, s).factor_total) + q_extra_bytes<float>(m, s);
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
