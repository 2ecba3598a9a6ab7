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

// The same back substitution for an FP32 right-hand side (the mixed-precision ID's W) in
// float-float arithmetic on the FP32 pipes, whose rate on this GPU is ~70x the FP64 rate:
// every value is an unevaluated sum hi + lo of two floats (~44 significant bits), R is given
// as such pairs (Rh, Rl, from the FP64 R), products are split exactly by FMA and sums kept by
// two-sum.  The result is far more accurate than the
// FP32 W it starts from.
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah + al) += (bh + bl) * (ch + cl), the lo * lo term dropped
__device__ __forceinline__ void ff_fma(float& ah, float& al, float bh, float bl, float ch, float cl) {
  const float p = __fmul_rn(bh, ch);
  float e = fmaf(bh, ch, -p);
  e = fmaf(bh, cl, e);
  e = fmaf(bl, ch, e);
  float sh, se;
  ff_two_sum(ah, p, sh, se);
  ah = sh;
  al = __fadd_rn(al, __fadd_rn(se, e));
}
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// Rows are solved in blocks of RB = 32 from the bottom: the off-diagonal update from the rows
// already solved (dot products over q >= hi, four independent float-float accumulators per
// thread), then the block's rows times the FP64 inverse of the 32 x 32 diagonal block (given
// as float pairs Dh, Dl: a product, parallel over rows and columns, instead of a sequential
// substitution).
__global__ void __launch_bounds__(256) trsm_upper_ff_kernel(int s, int64_t N, int nb, const float* Rh,
                                                            const float* Rl, const float* Dh, const float* Dl,
                                                            const float* B, int64_t ldb, double* Y, int64_t ldy) {
  extern __shared__ float Yff[];      // Yh [s][nb], then Yl [s][nb]
  float* Yh = Yff;
  float* Yl = Yff + (size_t)s * nb;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * nb;
  const int nc = (int)std::min<int64_t>(nb, N - c0);
  for (int64_t e = tid; e < (int64_t)s * nb; e += bd) {
    const int r = (int)(e / nb), cc = (int)(e % nb);
    Yh[e] = cc < nc ? B[(int64_t)r * ldb + c0 + cc] : 0.f;
    Yl[e] = 0.f;
  }
  __syncthreads();
  for (int kb = (s + RB - 1) / RB - 1; kb >= 0; --kb) {   // row blocks [32 kb, 32 kb + 32), last first
    const int lo = kb * RB, hi = std::min(s, lo + RB);
    // y(r) -= sum_{q >= hi} R(r, q) y(q), r in [lo, hi)
    if (hi < s)
      for (int e = tid; e < (hi - lo) * nb; e += bd) {
        const int r = lo + e / nb, cc = e % nb;
        const float* rh = Rh + (int64_t)r * s;
        const float* rl = Rl + (int64_t)r * s;
        float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
        int q = hi;
        for (; q + 3 < s; q += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            ff_fma(ah[u], al[u], __ldg(rh + q + u), __ldg(rl + q + u), Yh[(q + u) * nb + cc], Yl[(q + u) * nb + cc]);
        }
        for (; q < s; ++q) ff_fma(ah[0], al[0], __ldg(rh + q), __ldg(rl + q), Yh[q * nb + cc], Yl[q * nb + cc]);
        float h, l, t;
        ff_two_sum(ah[0], ah[1], h, t);
        l = __fadd_rn(__fadd_rn(al[0], al[1]), t);
        float h2, l2;
        ff_two_sum(ah[2], ah[3], h2, t);
        l2 = __fadd_rn(__fadd_rn(al[2], al[3]), t);
        float hs, ts;
        ff_two_sum(h, h2, hs, ts);
        const float ls = __fadd_rn(__fadd_rn(l, l2), ts);
        // Y(r) -= (hs + ls)
        const int idx = r * nb + cc;
        float sh, se;
        ff_two_sum(Yh[idx], -hs, sh, se);
        float lo2 = __fadd_rn(__fsub_rn(Yl[idx], ls), se);
        ff_norm(sh, lo2);
        Yh[idx] = sh;
        Yl[idx] = lo2;
      }
    __syncthreads();
    // y(lo:hi) = D_kb^{-1} y(lo:hi): D^{-1} upper triangular, rows of the block over threads
    const float* dh = Dh + (size_t)kb * RB * RB;
    const float* dl = Dl + (size_t)kb * RB * RB;
    const int nr = hi - lo;
    float zh[2], zl[2];
    for (int k = 0; k < 2; ++k) {
      const int e = tid + k * bd;
      zh[k] = 0.f;
      zl[k] = 0.f;
      if (e < nr * nb) {
        const int i = e / nb, cc = e % nb;
        for (int q = i; q < nr; ++q)
          ff_fma(zh[k], zl[k], dh[i * RB + q], dl[i * RB + q], Yh[(lo + q) * nb + cc], Yl[(lo + q) * nb + cc]);
        ff_norm(zh[k], zl[k]);
      }
    }
    __syncthreads();
    for (int k = 0; k < 2; ++k) {
      const int e = tid + k * bd;
      if (e < nr * nb) {
        Yh[lo * nb + e] = zh[k];
        Yl[lo * nb + e] = zl[k];
      }
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)s * nb; e += bd) {
    const int r = (int)(e / nb), cc = (int)(e % nb);
    if (cc < nc) Y[(int64_t)r * ldy + c0 + cc] = (double)Yh[e] + (double)Yl[e];
  }
}

// R (FP64, upper triangular) as float pairs, and the FP64 inverses of its RB x RB diagonal
// blocks as float pairs (block k at D + k RB^2, row-major; rows past s: the identity).
__global__ void ff_split_kernel(int s, const double* R, int64_t ldr, float* Rh, float* Rl) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / s), q = (int)(e % s);
    const double v = q >= r ? R[(int64_t)r * ldr + q] : 0.0;
    const float h = (float)v;
    Rh[e] = h;
    Rl[e] = (float)(v - (double)h);
  }
}

// One warp per diagonal block: lane j solves D x = e_j by back substitution in FP64.
__global__ void ff_diag_inverse_kernel(int s, const double* R, int64_t ldr, float* Dh, float* Dl) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nbk = (s + RB - 1) / RB;
  if (k >= nbk) return;
  const int b0 = RB * k;
  double x[RB];
#pragma unroll
  for (int i = RB - 1; i >= 0; --i) {
    double v;
    if (b0 + i >= s) {
      v = i == lane ? 1.0 : 0.0;
    } else {
      double acc = i == lane ? 1.0 : 0.0;
#pragma unroll
      for (int q = i + 1; q < RB; ++q)
        if (b0 + q < s) acc -= R[(int64_t)(b0 + i) * ldr + b0 + q] * x[q];
      v = acc / R[(int64_t)(b0 + i) * ldr + b0 + i];
    }
    x[i] = v;
  }
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const float h = (float)x[i];
    Dh[(size_t)k * RB * RB + i * RB + lane] = h;
    Dl[(size_t)k * RB * RB + i * RB + lane] = (float)(x[i] - (double)h);
  }
}

// Few right-hand sides (N small against the GPU): a CTA solves nbs = 4 columns.  The 32 x 32
// diagonal blocks of R are inverted first (warp k inverts block k by back substitution on the
// identity), so that the back substitution over the s/32 row blocks is, per block, one
// off-diagonal update (each warp owns 4 rows, its lanes split the dot products, a transposed
// shuffle reduction combines them) and one 32 x 32 upper triangular product.  Sequential depth
// s/32 instead of s.
constexpr int TS_NB = 4;
constexpr int TS_THREADS = 256;

template <int NV>
__device__ __forceinline__ void xreduce_d(double (&a)[NV], int lane) {
#pragma unroll
  for (int L = 0; L < 5; ++L) {
    const int m = 16 >> L;
    const int h = NV >> (L + 1);
    const bool up = (lane & m) != 0;
    if (h >= 1) {
#pragma unroll
      for (int k = 0; k < (NV >> (L + 1) > 0 ? NV >> (L + 1) : 1); ++k) {
        const double keep = up ? a[k + h] : a[k];
        const double send = up ? a[k] : a[k + h];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, m);
      }
    } else {
      a[0] += __shfl_xor_sync(0xffffffffu, a[0], m);
    }
  }
}

template <typename TB>
__global__ void __launch_bounds__(TS_THREADS) trsm_small_kernel(int s, int64_t N, const double* R, int64_t ldr,
                                                                int unit, const TB* B, int64_t ldb, double* Y,
                                                                int64_t ldy) {
  extern __shared__ double sm[];
  const int nbk = (s + 31) / 32;
  double* Dinv = sm;                                   // [nbk][32][32], row-major blocks
  double* Ys = Dinv + (size_t)nbk * 1024;              // [s][TS_NB]
  double* Tmp = Ys + (size_t)s * TS_NB;                // [32][TS_NB]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * TS_NB;
  const int nc = (int)std::min<int64_t>(TS_NB, N - c0);
  for (int e = tid; e < s * TS_NB; e += TS_THREADS) {
    const int r = e / TS_NB, cc = e % TS_NB;
    Ys[e] = cc < nc ? (double)B[(int64_t)r * ldb + c0 + cc] : 0.0;
  }
  // inverse of each diagonal block: lane j solves R_kk x = e_j (rows beyond s: identity)
  for (int k = warp; k < nbk; k += TS_THREADS / 32) {
    const int b0 = 32 * k;
    double* D = Dinv + (size_t)k * 1024;
    const int j = lane;
    for (int i = 31; i >= 0; --i) {
      double x;
      if (b0 + i >= s) {
        x = i == j ? 1.0 : 0.0;
      } else {
        double acc = i == j ? 1.0 : 0.0;
        for (int q = i + 1; q < 32 && b0 + q < s; ++q) acc -= __ldg(R + (int64_t)(b0 + i) * ldr + b0 + q) * D[q * 32 + j];
        x = unit ? acc : acc / __ldg(R + (int64_t)(b0 + i) * ldr + b0 + i);
      }
      D[i * 32 + j] = x;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = nbk - 1; k >= 0; --k) {
    const int b0 = 32 * k;
    const int qlo = b0 + 32;
    if (qlo < s) {
      // Y_k -= R(k-block, qlo:) Y(qlo:, :): warp w owns rows b0+4w .. +3; lanes split q
      double a[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) a[e] = 0.0;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int r = b0 + 4 * warp + rr;
        if (r >= s) continue;
        const double* Rr = R + (int64_t)r * ldr;
        for (int q = qlo + lane; q < s; q += 32) {
          const double rq = __ldg(Rr + q);
#pragma unroll
          for (int cc = 0; cc < TS_NB; ++cc) a[rr * TS_NB + cc] = fma(rq, Ys[q * TS_NB + cc], a[rr * TS_NB + cc]);
        }
      }
      xreduce_d<16>(a, lane);
      if ((lane & 1) == 0) {
        int idx = 0;
#pragma unroll
        for (int L = 0; L < 4; ++L)
          if (lane & (16 >> L)) idx += 16 >> (L + 1);
        const int r = b0 + 4 * warp + idx / TS_NB, cc = idx % TS_NB;
        if (r < s) Ys[r * TS_NB + cc] -= a[0];
      }
      __syncthreads();
    }
    // Y_k = inv(R_kk) Y_k
    if (tid < 32 * TS_NB) {
      const int i = tid / TS_NB, cc = tid % TS_NB;
      const double* D = Dinv + (size_t)k * 1024 + i * 32;
      double acc = 0.0;
      for (int q = i; q < 32 && b0 + q < s; ++q) acc = fma(D[q], Ys[(b0 + q) * TS_NB + cc], acc);
      Tmp[tid] = acc;
    }
    __syncthreads();
    if (tid < 32 * TS_NB) {
      const int i = tid / TS_NB;
      if (b0 + i < s) Ys[(b0 + i) * TS_NB + tid % TS_NB] = Tmp[tid];
    }
    __syncthreads();
  }
  for (int e = tid; e < s * TS_NB; e += TS_THREADS) {
    const int r = e / TS_NB, cc = e % TS_NB;
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

// U(i, j) = R(s-1-j, s-1-i) for j >= i, 0 below: with J the order-reversing permutation,
// U = J R^T J is upper triangular, and R^T Y = D is U (J Y) = J D.
__global__ void flip_transpose_kernel(int s, const double* R, int64_t ldr, double* U, int64_t ldu) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / s), j = (int)(e % s);
    U[(int64_t)i * ldu + j] = j >= i ? R[(int64_t)(s - 1 - j) * ldr + (s - 1 - i)] : 0.0;
  }
}

// Z(r, :) += X(r, :) for the rows r = blockIdx.y (+ gridDim.y ...), coalesced along each row.
template <typename T>
__global__ void axpy_rows_kernel(int s, int64_t n, const T* X, int64_t ldx, T* Z, int64_t ldz) {
  for (int64_t r = blockIdx.y; r < s; r += gridDim.y) {
    const T* x = X + r * ldx;
    T* z = Z + r * ldz;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
      z[c] += x[c];
  }
}

template <typename T>
cudaError_t launch_axpy_rows_t(int32_t s, int64_t n, const T* X, int64_t ldx, T* Z, int64_t ldz, cudaStream_t st) {
  if (s <= 0 || n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<int64_t>((n + 1023) / 1024, 64), (unsigned)std::min<int32_t>(s, 65535));
  axpy_rows_kernel<T><<<grid, 256, 0, st>>>(s, n, X, ldx, Z, ldz);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trsm_upper_t(int32_t s, int64_t N, const double* R, int64_t ldr, double* U, double* D,
                                int64_t ldd, cudaStream_t st) {
  if (N <= 0 || s <= 0) return cudaSuccess;
  flip_transpose_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * s + 255) / 256, 1024), 256, 0, st>>>(s, R, ldr,
                                                                                                        U, s);
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
  // rows taken from the last one up (negative leading dimension): J D in, J Y out
  double* last = D + (int64_t)(s - 1) * ldd;
  return launch_trsm_upper(s, N, U, s, 0, SKEL_F64, last, -ldd, last, -ldd, st);
}

cudaError_t launch_axpy_rows_f64(int32_t s, int64_t n, const double* X, int64_t ldx, double* Z, int64_t ldz,
                                 cudaStream_t st) {
  return launch_axpy_rows_t<double>(s, n, X, ldx, Z, ldz, st);
}

cudaError_t launch_axpy_rows_f32(int32_t s, int64_t n, const float* X, int64_t ldx, float* Z, int64_t ldz,
                                 cudaStream_t st) {
  return launch_axpy_rows_t<float>(s, n, X, ldx, Z, ldz, st);
}

cudaError_t launch_trsm_upper(int32_t s, int64_t N, const double* R, int64_t ldr, int unit_diag,
                              skel_dtype b_dt, const void* B, int64_t ldb, double* Y, int64_t ldy,
                              cudaStream_t st) {
  if (N <= 0 || s <= 0) return cudaSuccess;
  const int sms = device_sm_count();
  const size_t small_smem = sizeof(double) * ((size_t)((s + 31) / 32) * 1024 + (size_t)s * TS_NB + 32 * TS_NB);
  if ((N + TS_NB - 1) / TS_NB <= 4 * sms && small_smem <= 200 * 1024) {
    KernelTimer kt("trsm", st);
    cudaError_t e;
    const unsigned grid = (unsigned)((N + TS_NB - 1) / TS_NB);
    if (b_dt == SKEL_F64) {
      e = cudaFuncSetAttribute(trsm_small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem);
      if (e != cudaSuccess) return e;
      trsm_small_kernel<double><<<grid, TS_THREADS, small_smem, st>>>(s, N, R, ldr, unit_diag, (const double*)B, ldb, Y, ldy);
    } else {
      e = cudaFuncSetAttribute(trsm_small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem);
      if (e != cudaSuccess) return e;
      trsm_small_kernel<float><<<grid, TS_THREADS, small_smem, st>>>(s, N, R, ldr, unit_diag, (const float*)B, ldb, Y, ldy);
    }
    note_launches(1);
    return cudaGetLastError();
  }
  int nb = 32;
  while (nb > 2 && (N + nb - 1) / nb < 2 * sms) nb >>= 1;
  while ((size_t)s * nb * sizeof(double) > 160 * 1024 && nb > 1) nb >>= 1;
  const size_t smem = (size_t)s * nb * sizeof(double);
  const unsigned grid = (unsigned)((N + nb - 1) / nb);
  cudaError_t e;
  KernelTimer kt("trsm", st);
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

size_t trsm_ff_workspace(int32_t s) {
  const size_t nbk = (size_t)(s + RB - 1) / RB;
  return 2 * align_up(sizeof(float) * (size_t)s * s) + 2 * align_up(sizeof(float) * nbk * RB * RB);
}

cudaError_t launch_trsm_upper_ff(int32_t s, int64_t N, const double* R, int64_t ldr, const float* B, int64_t ldb,
                                 double* Y, int64_t ldy, void* ws, cudaStream_t st) {
  if (N <= 0 || s <= 0) return cudaSuccess;
  char* base = static_cast<char*>(ws);
  float* Rh = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * (size_t)s * s);
  float* Rl = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * (size_t)s * s);
  const size_t nbk = (size_t)(s + RB - 1) / RB;
  float* Dh = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * nbk * RB * RB);
  float* Dl = reinterpret_cast<float*>(base);
  ff_split_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * s + 255) / 256, 4096), 256, 0, st>>>(s, R, ldr, Rh, Rl);
  ff_diag_inverse_kernel<<<(unsigned)((nbk + 3) / 4), 128, 0, st>>>(s, R, ldr, Dh, Dl);
  note_launches(2);
  const int sms = device_sm_count();
  // eight columns per CTA (~64 KB of shared memory at s = 1024: three CTAs per SM) unless
  // that leaves too few CTAs
  int nb = 8;
  while (nb > 2 && (N + nb - 1) / nb < 2 * sms) nb >>= 1;
  while ((size_t)s * nb * 2 * sizeof(float) > 160 * 1024 && nb > 1) nb >>= 1;
  const size_t smem = (size_t)s * nb * 2 * sizeof(float);
  const cudaError_t e = cudaFuncSetAttribute(trsm_upper_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  {
    KernelTimer kt("trsm_ff", st);
    trsm_upper_ff_kernel<<<(unsigned)((N + nb - 1) / nb), 256, smem, st>>>(s, N, nb, Rh, Rl, Dh, Dl, B, ldb, Y, ldy);
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
    a.timer = "gemm_eta_sq";
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
