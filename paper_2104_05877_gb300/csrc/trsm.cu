// FP64 triangular solves (Z = R_C^{-1} W for Eq. (2.1); U = R_C^{-1} M R_R^{-T} for Remark 3;
// R_1^{-1} ... for Theorem 1's eta) and the largest-eigenvalue routine behind eta.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int RB = 32;    // row block of the back substitution

template <typename TB>
__global__ void __launch_bounds__(256) trsm_upper_kernel(int s, int64_t N, int nb, const double* R,
                                                         int64_t ldr, int unit, const TB* B,
                                                         int64_t ldb, double* Y, int64_t ldy) {
  extern __shared__ double Ys[];     // [s][nb]
  const int tid = threadIdx.x, bd = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * nb;
  const int nc = (int)std::min<int64_t>(nb, N - c0);
  for (int64_t e = tid; e < (int64_t)s * nb; e += bd) {
    const int r = (int)(e / nb), cc = (int)(e % nb);
    Ys[e] = cc < nc ? (double)B[(int64_t)r * ldb + c0 + cc] : 0.0;
  }
  __syncthreads();
  for (int hi = s; hi > 0; hi -= RB) {
    const int lo = std::max(0, hi - RB);
    // off-diagonal update from the solved rows q >= hi: one thread per (row, column) pair
    if (hi < s) {
      for (int e = tid; e < (hi - lo) * nb; e += bd) {
        const int r = lo + e / nb, cc = e % nb;
        const double* Rr = R + (int64_t)r * ldr;
        double acc = 0.0;
        for (int q = hi; q < s; ++q) acc = fma(__ldg(Rr + q), Ys[q * nb + cc], acc);
        Ys[r * nb + cc] -= acc;
      }
      __syncthreads();
    }
    // diagonal block: rows hi-1 .. lo in order, threads over columns
    for (int r = hi - 1; r >= lo; --r) {
      const double* Rr = R + (int64_t)r * ldr;
      for (int cc = tid; cc < nb; cc += bd) {
        double acc = Ys[r * nb + cc];
        for (int q = r + 1; q < hi; ++q) acc -= __ldg(Rr + q) * Ys[q * nb + cc];
        Ys[r * nb + cc] = unit ? acc : acc / __ldg(Rr + r);
      }
      __syncthreads();
    }
  }
  for (int64_t e = tid; e < (int64_t)s * nb; e += bd) {
    const int r = (int)(e / nb), cc = (int)(e % nb);
    if (cc < nc) Y[(int64_t)r * ldy + c0 + cc] = Ys[e];
  }
}

// Normalise an s x s matrix by its trace: M /= tr(M); logs[slot] = log(tr(M)).
__global__ void trace_normalize_kernel(int s, double* M, int64_t ldm, double* logs, int slot) {
  double v = 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) v += M[(int64_t)i * ldm + i];
  v = block_sum<double>(v);
  const double inv = v > 0.0 ? 1.0 / v : 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)s * s; e += blockDim.x) M[(e / s) * ldm + e % s] *= inv;
  if (threadIdx.x == 0) logs[slot] = log(v);
}

// Power iteration on a symmetric s x s matrix N (trace 1) -> logs[slot] = log(lambda_max(N)).
__global__ void __launch_bounds__(1024) power_kernel(int s, const double* N, int64_t ldn,
                                                     double* logs, int slot, int maxit) {
  __shared__ double x[kMaxS];
  __shared__ double y[kMaxS];
  __shared__ int s_done;
  const int tid = threadIdx.x;
  for (int i = tid; i < s; i += blockDim.x) x[i] = 1.0 / sqrt((double)s) * (1.0 + 1e-3 * (i % 7));
  if (tid == 0) s_done = 0;
  __syncthreads();
  double lam = 0.0, lam_prev = -1.0;
  for (int it = 0; it < maxit; ++it) {
    double nx = 0.0;
    for (int i = tid; i < s; i += blockDim.x) nx += x[i] * x[i];
    nx = block_sum<double>(nx);
    const double inv = 1.0 / sqrt(nx);
    for (int i = tid; i < s; i += blockDim.x) {
      const double* Nr = N + (int64_t)i * ldn;
      double acc = 0.0;
      for (int q = 0; q < s; ++q) acc = fma(__ldg(Nr + q), x[q], acc);
      y[i] = acc * inv;
    }
    __syncthreads();
    double rq = 0.0;
    for (int i = tid; i < s; i += blockDim.x) rq += x[i] * inv * y[i];
    lam = block_sum<double>(rq);
    for (int i = tid; i < s; i += blockDim.x) x[i] = y[i];
    if (tid == 0 && fabs(lam - lam_prev) <= 1e-13 * fabs(lam)) s_done = 1;
    __syncthreads();
    if (s_done) break;
    lam_prev = lam;
  }
  if (tid == 0) logs[slot] = log(lam);
}

// lambda(N_0) = exp((log lambda(N_q) + sum_i 2^(q-i) log c_i) / 2^q) * c_0, eta = sqrt(.)
__global__ void eta_finalize_kernel(const double* logs, int q, double* out) {
  if (threadIdx.x != 0) return;
  double acc = logs[q + 1];                 // log lambda(N_q)
  for (int i = 1; i <= q; ++i) acc += ldexp(1.0, q - i) * logs[i];
  const double log_lam = acc / ldexp(1.0, q) + logs[0];
  *out = sqrt(exp(log_lam));
}

}  // namespace

cudaError_t launch_trsm_upper(int32_t s, int64_t N, const double* R, int64_t ldr, int unit_diag,
                              skel_dtype b_dt, const void* B, int64_t ldb, double* Y, int64_t ldy,
                              cudaStream_t st) {
  if (N <= 0 || s <= 0) return cudaSuccess;
  const int sms = device_sm_count();
  int nb = 32;
  while (nb > 2 && (N + nb - 1) / nb < 2 * sms) nb >>= 1;
  while ((size_t)s * nb * sizeof(double) > 160 * 1024 && nb > 1) nb >>= 1;
  const size_t smem = (size_t)s * nb * sizeof(double);
  const unsigned grid = (unsigned)((N + nb - 1) / nb);
  cudaError_t e;
  if (b_dt == SKEL_F64) {
    e = cudaFuncSetAttribute(trsm_upper_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    trsm_upper_kernel<double><<<grid, 256, smem, st>>>(s, N, nb, R, ldr, unit_diag, (const double*)B, ldb, Y, ldy);
  } else {
    e = cudaFuncSetAttribute(trsm_upper_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    trsm_upper_kernel<float><<<grid, 256, smem, st>>>(s, N, nb, R, ldr, unit_diag, (const float*)B, ldb, Y, ldy);
  }
  note_launches(1);
  return cudaGetLastError();
}

// sqrt(lambda_max(M)) for a symmetric positive definite s x s M (overwritten).  M is
// normalised by its trace and squared q times (N_i = N_{i-1}^2 / tr(N_{i-1}^2)), so that the
// power iteration sees the eigenvalue ratio raised to the 2^q-th power.
size_t power_scratch_bytes(int32_t s) {
  return align_up(sizeof(double) * (16 + 2 * (size_t)s * s)) + gemm_workspace(s, s, s, true);
}

cudaError_t launch_power_sqrt_lmax(int32_t s, const double* Min, int64_t ldm, double* out,
                                   double* scratch, cudaStream_t st) {
  // scratch layout: [logs: 16 doubles][two s x s buffers][split-K scratch]
  constexpr int q = 4;
  double* logs = scratch;
  double* bufA = scratch + 16;
  double* bufB = bufA + (int64_t)s * s;
  void* kws = reinterpret_cast<char*>(scratch) + align_up(sizeof(double) * (16 + 2 * (size_t)s * s));
  cudaError_t e = cudaMemcpy2DAsync(bufA, sizeof(double) * s, Min, sizeof(double) * ldm,
                                    sizeof(double) * s, s, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  trace_normalize_kernel<<<1, 1024, 0, st>>>(s, bufA, s, logs, 0);
  double* cur = bufA;
  double* nxt = bufB;
  for (int i = 1; i <= q; ++i) {
    GemmArgs a{};
    a.M = s; a.N = s; a.K = s;
    a.L = View{cur, s, 1}; a.l_dt = SKEL_F64;
    a.B = View{cur, s, 1}; a.b_dt = SKEL_F64;      // symmetric: B(k, c) = cur(k, c)
    a.out = nxt; a.out_sr = s; a.out_sc = 1; a.out_dt = SKEL_F64;
    a.alpha = 1.0;
    a.splitk_ws = gemm_workspace(s, s, s, true) ? kws : nullptr;
    e = launch_gemm(a, true, LEFT_LOAD, EPI_STORE, st);
    if (e != cudaSuccess) return e;
    trace_normalize_kernel<<<1, 1024, 0, st>>>(s, nxt, s, logs, i);
    std::swap(cur, nxt);
  }
  power_kernel<<<1, 1024, 0, st>>>(s, cur, s, logs, q + 1, 300);
  eta_finalize_kernel<<<1, 32, 0, st>>>(logs, q, out);
  note_launches(3 + q);
  return cudaGetLastError();
}

}  // namespace skel
