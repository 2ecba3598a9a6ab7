// SIMT tiled GEMM with pluggable left operand (loaded, or Gaussian generated in-kernel from
// Philox) and fused epilogues; plus gathers, transposes and deterministic reductions.
//
// Used for: the FP64/FP32 Gaussian sketch X = Gamma A (Algorithm 2, sketch step) with Gamma never
// stored; W = Q_C^T A (Eq. (2.1) via Q_C R_C = C); W Q_R (Remark 3); T T^T for Theorem 1's
// eta; and the residual norms ||A - C Z||_F, ||A - C U R||_F.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int BM = 64, BN = 128, BK = 16, NT = 256;
constexpr int TM = 4, TN = 8;   // per-thread micro tile: rows ty*4+i, cols tx+16*j

template <typename T>
__device__ __forceinline__ T load_as(const void* p, int64_t off, skel_dtype dt) {
  return dt == SKEL_F64 ? (T)__ldg(static_cast<const double*>(p) + off)
                        : (T)__ldg(static_cast<const float*>(p) + off);
}

template <typename T, int LEFT, int EPI, bool SPLIT>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmArgs a) {
  __shared__ T Ls[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)blockIdx.y * BM, c0 = (int64_t)blockIdx.x * BN;
  const uint32_t k0s = (uint32_t)(a.seed & 0xffffffffu), k1s = (uint32_t)(a.seed >> 32);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  const bool l_kcontig = (a.L.sc == 1);
  const bool b_kcontig = (a.B.sr == 1);
  const int64_t kz0 = (int64_t)blockIdx.z * a.kchunk;
  const int64_t kz1 = kz0 + a.kchunk < a.K ? kz0 + a.kchunk : a.K;
  // Loaded operands: the next K-tile is fetched into registers while the current one is used
  // (one tile of global-load latency hidden per step); the Gaussian left operand is generated
  // straight into shared memory.
  constexpr int LPT = BM * BK / NT, BPT = BK * BN / NT;   // elements per thread: 4, 8
  T lreg[LPT], breg[BPT];
  auto fetch = [&](int64_t kb) {
    if (LEFT != LEFT_GAUSSIAN) {
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        const int e = q * NT + tid;
        int r, k;
        if (l_kcontig) { r = e / BK; k = e % BK; } else { r = e % BM; k = e / BM; }
        const int64_t gr = r0 + r, gk = kb + k;
        lreg[q] = (gr < a.M && gk < kz1) ? load_as<T>(a.L.p, gr * a.L.sr + gk * a.L.sc, a.l_dt) : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int e = q * NT + tid;
      int k, c;
      if (b_kcontig) { k = e % BK; c = e / BK; } else { c = e % BN; k = e / BN; }
      const int64_t gk = kb + k, gc = c0 + c;
      breg[q] = (gk < kz1 && gc < a.N) ? load_as<T>(a.B.p, gk * a.B.sr + gc * a.B.sc, a.b_dt) : T(0);
    }
  };
  if (kz0 < kz1) fetch(kz0);
  for (int64_t kb = kz0; kb < kz1; kb += BK) {
    // ---- left tile (BM x BK) ----
    if (LEFT == LEFT_GAUSSIAN) {
      const int r = tid >> 2, k4 = tid & 3;       // 64 rows x 4 groups of 4 columns
      const int64_t gr = r0 + r;
      const int64_t gk = kb + 4 * k4;
      T g[4] = {T(0), T(0), T(0), T(0)};
      if (gr < a.M && gk < a.K) {
        if constexpr (sizeof(T) == 8) {
          double d[4];
          gaussian4_f64(k0s, k1s, (uint32_t)gr, (uint32_t)((a.gcol0 + gk) >> 2), d);
#pragma unroll
          for (int q = 0; q < 4; ++q) g[q] = (T)d[q];
        } else {
          const float4 f = gaussian4_f32(k0s, k1s, (uint32_t)gr, (uint32_t)((a.gcol0 + gk) >> 2));
          g[0] = f.x; g[1] = f.y; g[2] = f.z; g[3] = f.w;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) Ls[4 * k4 + q][r] = (gk + q < a.K) ? g[q] : T(0);
    } else {
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        const int e = q * NT + tid;
        int r, k;
        if (l_kcontig) { r = e / BK; k = e % BK; } else { r = e % BM; k = e / BM; }
        Ls[k][r] = lreg[q];
      }
    }
    // ---- right tile (BK x BN) ----
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int e = q * NT + tid;
      int k, c;
      if (b_kcontig) { k = e % BK; c = e / BK; } else { c = e % BN; k = e / BN; }
      Bs[k][c] = breg[q];
    }
    __syncthreads();
    if (kb + BK < kz1) fetch(kb + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T lv[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) lv[i] = Ls[k][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(lv[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  // ---- epilogue ----
  if (SPLIT) {        // raw partial sums of this K-chunk: ws[z][r][c]
    T* ws = static_cast<T*>(a.splitk_ws) + (int64_t)blockIdx.z * a.M * a.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gr = r0 + ty * TM + i;
      if (gr >= a.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gc = c0 + tx + 16 * j;
        if (gc < a.N) ws[gr * a.N + gc] = acc[i][j];
      }
    }
    return;
  }
  const T alpha = (T)a.alpha;
  double part = 0.0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gr = r0 + ty * TM + i;
    if (gr >= a.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gc = c0 + tx + 16 * j;
      if (gc >= a.N) continue;
      const T v = alpha * acc[i][j];
      if (EPI == EPI_RESID) {
        const double d = load_as<double>(a.ref.p, gr * a.ref.sr + gc * a.ref.sc, a.ref_dt) - (double)v;
        part += d * d;
      } else if (EPI == EPI_ACCUM) {
        const int64_t off = gr * a.out_sr + gc * a.out_sc;
        if (a.out_dt == SKEL_F64) static_cast<double*>(a.out)[off] += (double)v;
        else static_cast<float*>(a.out)[off] += (float)v;
      } else {
        const int64_t off = gr * a.out_sr + gc * a.out_sc;
        if (a.out_dt == SKEL_F64) static_cast<double*>(a.out)[off] = (double)v;
        else static_cast<float*>(a.out)[off] = (float)v;
        if (EPI == EPI_STORE_SQ) part += (double)v * (double)v;
        if (EPI == EPI_SKETCH && !isfinite(v)) bad = true;
      }
    }
  }
  if (EPI == EPI_SKETCH && bad) record_error(a.dev_status, SKEL_ERR_NONFINITE, -1);
  if (EPI == EPI_RESID || EPI == EPI_STORE_SQ) {
    const double tot = block_sum<double>(part);
    if (tid == 0) a.partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

// Sum the K-chunk partials in chunk order, then apply the STORE / STORE_SQ epilogue.  The
// grid has gemm_num_blocks(M, N) CTAs so that STORE_SQ writes as many partials as the
// unsplit kernel.
template <typename T, int EPI>
__global__ void __launch_bounds__(NT) splitk_reduce_kernel(const GemmArgs a, int nz) {
  const T* ws = static_cast<const T*>(a.splitk_ws);
  const int64_t total = a.M * a.N;
  double part = 0.0;
  // rows of the output are dealt to CTAs, columns to threads
  for (int64_t r = blockIdx.x; r < a.M; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < a.N; c += blockDim.x) {
      const int64_t e = r * a.N + c;
      T acc = T(0);
      for (int z = 0; z < nz; ++z) acc += ws[(int64_t)z * total + e];
      const T v = (T)a.alpha * acc;
      const int64_t off = r * a.out_sr + c * a.out_sc;
      if (a.out_dt == SKEL_F64) static_cast<double*>(a.out)[off] = (double)v;
      else static_cast<float*>(a.out)[off] = (float)v;
      if (EPI == EPI_STORE_SQ) part += (double)v * (double)v;
    }
  if (EPI == EPI_STORE_SQ) {
    const double tot = block_sum<double>(part);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
  }
}

template <typename T, int LEFT, int EPI>
cudaError_t launch_t(const GemmArgs& a0, int nz, cudaStream_t st) {
  GemmArgs a = a0;
  const unsigned gx = (unsigned)((a.N + BN - 1) / BN), gy = (unsigned)((a.M + BM - 1) / BM);
  if (nz > 1 && (EPI == EPI_STORE || EPI == EPI_STORE_SQ) && LEFT == LEFT_LOAD) {
    {
      KernelTimer kt(a.timer ? a.timer : "gemm_simt", st);
      gemm_kernel<T, LEFT, EPI, true><<<dim3(gx, gy, nz), NT, 0, st>>>(a);
    }
    // STORE_SQ writes one partial per reduce CTA, so it keeps the tile count as its grid
    const int64_t total = a.M * a.N;
    const unsigned rg = EPI == EPI_STORE_SQ ? gx * gy
                        : (unsigned)std::max<int64_t>(gx * gy, std::min<int64_t>((total + NT - 1) / NT, 1024));
    splitk_reduce_kernel<T, EPI><<<rg, NT, 0, st>>>(a, nz);
    note_launches(2);
  } else {
    a.kchunk = a.K;
    {
      KernelTimer kt(a.timer ? a.timer : "gemm_simt", st);
      gemm_kernel<T, LEFT, EPI, false><<<dim3(gx, gy, 1), NT, 0, st>>>(a);
    }
    note_launches(1);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_epi(const GemmArgs& a, int nz, GemmLeft left, GemmEpi epi, cudaStream_t st) {
  if (left == LEFT_GAUSSIAN) {
    if (epi == EPI_SKETCH) return launch_t<T, LEFT_GAUSSIAN, EPI_SKETCH>(a, 1, st);
    return cudaErrorInvalidValue;
  }
  switch (epi) {
    case EPI_STORE: return launch_t<T, LEFT_LOAD, EPI_STORE>(a, nz, st);
    case EPI_STORE_SQ: return launch_t<T, LEFT_LOAD, EPI_STORE_SQ>(a, nz, st);
    case EPI_RESID: return launch_t<T, LEFT_LOAD, EPI_RESID>(a, 1, st);
    case EPI_SKETCH: return launch_t<T, LEFT_LOAD, EPI_SKETCH>(a, 1, st);
    case EPI_ACCUM: return launch_t<T, LEFT_LOAD, EPI_ACCUM>(a, 1, st);
  }
  return cudaErrorInvalidValue;
}

// H = R R^T (s x s, FP64) for an FP32 s x n row-major R with float-float accumulation: each
// product a*b is split exactly into p + e (p = a*b, e = fma(a, b, -p)) and added to a (hi, lo)
// pair by an error-free two-sum, which keeps ~44 significant bits on the FP32 pipes (FP64
// arithmetic is scarce on this GPU).  64 x 64 tiles of the upper triangle, the K range split
// into chunks; the chunk partials are summed in FP64 by syrk_ff_reduce_kernel.
constexpr int FF_T = 64, FF_BK = 16;
__device__ __forceinline__ void ff_add_prod(float a, float b, float& hi, float& lo) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = hi + p;
  const float z = t - hi;
  const float err = (hi - (t - z)) + (p - z);
  hi = t;
  lo += err + e;
}

__global__ void __launch_bounds__(256) syrk_ff_kernel(int s, int64_t n, const float* R, int64_t ldr,
                                                      int64_t kchunk, double* part) {
  __shared__ float As[FF_BK][FF_T + 4], Bs[FF_BK][FF_T + 4];
  // blockIdx.x enumerates the tile pairs ti <= tj
  int ti = 0, rem = blockIdx.x;
  const int nt = (s + FF_T - 1) / FF_T;
  while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
  const int tj = ti + rem;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t k0 = (int64_t)blockIdx.y * kchunk;
  const int64_t k1 = k0 + kchunk < n ? k0 + kchunk : n;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
  for (int64_t kb = k0; kb < k1; kb += FF_BK) {
#pragma unroll
    for (int q = 0; q < FF_T * FF_BK / 256; ++q) {
      const int e = q * 256 + tid;
      const int r = e / FF_BK, k = e % FF_BK;
      const int64_t gk = kb + k;
      const int ra = ti * FF_T + r, rb = tj * FF_T + r;
      As[k][r] = (ra < s && gk < k1) ? R[(int64_t)ra * ldr + gk] : 0.f;
      Bs[k][r] = (rb < s && gk < k1) ? R[(int64_t)rb * ldr + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < FF_BK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ff_add_prod(a[i], b[j], hi[i][j], lo[i][j]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * s * s;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ti * FF_T + ty * 4 + i, c = tj * FF_T + tx * 4 + j;
      if (r < s && c < s && c >= r) out[(int64_t)r * s + c] = (double)hi[i][j] + (double)lo[i][j];
    }
}

// out(r, c) = sum_k C(k, r) B(k, c) (s x n, FP64) for FP32 column-major C (m x s) and B
// (m x n), every product split exactly into p + e and accumulated in a float-float pair (the
// error-free transformations above): the products are exact and each sum keeps ~44 bits, on
// the FP32 pipes.  64 x 64 output tiles; the K range split into chunks whose FP64 partials are
// summed in chunk order (or, with one chunk, stored directly).
__global__ void __launch_bounds__(256) gemm_tn_ff_kernel(int s, int64_t n, int64_t m, const float* C, int64_t ldc,
                                                         const float* B, int64_t ldb, int64_t kchunk, double* out,
                                                         int64_t ldo, int64_t part_stride) {
  __shared__ float As[FF_BK][FF_T + 4], Bs[FF_BK][FF_T + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * FF_T;
  const int64_t c0 = (int64_t)blockIdx.x * FF_T;
  const int64_t k0 = (int64_t)blockIdx.z * kchunk;
  const int64_t k1 = k0 + kchunk < m ? k0 + kchunk : m;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
  for (int64_t kb = k0; kb < k1; kb += FF_BK) {
#pragma unroll
    for (int q = 0; q < FF_T * FF_BK / 256; ++q) {
      const int e = q * 256 + tid;
      const int r = e / FF_BK, k = e % FF_BK;
      const int64_t gk = kb + k;
      As[k][r] = (r0 + r < s && gk < k1) ? __ldg(C + gk + (int64_t)(r0 + r) * ldc) : 0.f;
      Bs[k][r] = (c0 + r < n && gk < k1) ? __ldg(B + gk + (c0 + r) * ldb) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < FF_BK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ff_add_prod(a[i], b[j], hi[i][j], lo[i][j]);
    }
    __syncthreads();
  }
  double* o = out + (int64_t)blockIdx.z * part_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i;
      const int64_t c = c0 + tx * 4 + j;
      if (r < s && c < n) o[(int64_t)r * ldo + c] = (double)hi[i][j] + (double)lo[i][j];
    }
}

// out(r, c) = sum_z part[z][r][c] in chunk order (s x n)
__global__ void ff_reduce_kernel(int s, int64_t n, int P, const double* part, double* out, int64_t ldo) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int z = 0; z < P; ++z) a += part[(int64_t)z * s * n + e];
    out[(e / n) * ldo + e % n] = a;
  }
}

// H(r, c) = H(c, r) = sum over chunks of part[z][r][c] (upper entries, chunk order)
__global__ void syrk_ff_reduce_kernel(int s, int P, const double* part, double* H, int64_t ldh) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / s), c = (int)(e % s);
    if (c < r) continue;
    double a = 0.0;
    for (int z = 0; z < P; ++z) a += part[(int64_t)z * s * s + e];
    H[(int64_t)r * ldh + c] = a;
    H[(int64_t)c * ldh + r] = a;
  }
}

// Z(r, Js[t]) = (r == t) for an s x ? row-major FP64 Z: the interpolation's identity columns.
__global__ void unit_columns_kernel(int32_t s, const int32_t* Js, double* Z, int64_t ldz) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / s), t = (int)(e % s);
    Z[(int64_t)r * ldz + Js[t]] = r == t ? 1.0 : 0.0;
  }
}

// ------------------------------------------------------------------------------------
__global__ void reduce_sum_kernel(const double* p, int64_t count, double* out, int take_sqrt) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) v += p[i];
  v = block_sum<double>(v);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(v) : v;
}

constexpr int SQ_COLS = 8;
// ||A||_F^2 partials, one per CTA (8 columns, fixed order).  FP32 data: 16-byte loads and
// squares summed in FP32 over 16 elements, then in FP64 (the FP32 roundings are unbiased and
// far below what the Gram-identity errors need); FP64 data: plain FP64.
template <typename T>
__global__ void __launch_bounds__(256) sqnorm_kernel(int64_t m, int64_t n, const T* A, int64_t lda,
                                                     double* partials) {
  double v = 0.0;
  const int64_t c0 = (int64_t)blockIdx.x * SQ_COLS;
  const bool vec = sizeof(T) == 4 && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  for (int cc = 0; cc < SQ_COLS; ++cc) {
    const int64_t c = c0 + cc;
    if (c >= n) break;
    const T* col = A + c * lda;
    if constexpr (sizeof(T) == 4) {
      if (vec) {
        const int64_t m4 = m / 4;
        const float4* c4 = reinterpret_cast<const float4*>(col);
        int64_t i = threadIdx.x;
        for (; i + 3 * 256 < m4; i += 4 * 256) {      // 16 elements per thread per pass
          float a = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 x = c4[i + u * 256];
            a = fmaf(x.x, x.x, a); a = fmaf(x.y, x.y, a); a = fmaf(x.z, x.z, a); a = fmaf(x.w, x.w, a);
          }
          v += (double)a;
        }
        for (; i < m4; i += 256) {
          const float4 x = c4[i];
          v += (double)(x.x * x.x + x.y * x.y) + (double)(x.z * x.z + x.w * x.w);
        }
        for (int64_t r = 4 * m4 + threadIdx.x; r < m; r += 256) v += (double)col[r] * col[r];
        continue;
      }
    }
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const double x = (double)col[i];
      v += x * x;
    }
  }
  v = block_sum<double>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// Quiet NaN of the element type: what a gather writes for an index outside the matrix (never
// reading it), so that the non-finite checks downstream report the bad index.
template <typename T> __device__ __forceinline__ T gather_nan();
template <> __device__ __forceinline__ float gather_nan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double gather_nan<double>() { return __longlong_as_double(0x7ff8000000000000ll); }

template <typename T>
__global__ void gather_cols_kernel(int64_t m, const T* A, int64_t lda, int64_t ncols, const int32_t* idx,
                                   T* C, int64_t ldc) {
  const int r = blockIdx.y;
  const int64_t src = (int64_t)idx[r];
  const bool ok = src >= 0 && src < ncols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    C[i + r * ldc] = ok ? A[i + src * lda] : gather_nan<T>();
}

template <typename T>
__global__ void gather_rows_t_kernel(int64_t n, int32_t s, const T* A, int64_t lda, int64_t nrows,
                                     const int32_t* idx, T* Rt, int64_t ldr) {
  const int r = blockIdx.y;
  const int64_t row = (int64_t)idx[r];
  const bool ok = row >= 0 && row < nrows;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    Rt[c + r * ldr] = ok ? A[row + c * lda] : gather_nan<T>();
}

__global__ void gather_cols_rm_kernel(int32_t s, skel_dtype dt, const void* F, int64_t ldf, int64_t ncols,
                                      const int32_t* idx, double* out, int64_t ldo) {
  const int r = blockIdx.x;
  for (int t = threadIdx.x; t < s; t += blockDim.x) {
    const int64_t j = idx[t];
    out[(int64_t)r * ldo + t] = j >= 0 && j < ncols ? load_as<double>(F, (int64_t)r * ldf + j, dt)
                                                    : gather_nan<double>();
  }
}

__global__ void transpose_kernel(int32_t s, const double* in, int64_t ldi, double* out, int64_t ldo) {
  const int r = blockIdx.x;
  for (int c = threadIdx.x; c < s; c += blockDim.x) out[(int64_t)c * ldo + r] = in[(int64_t)r * ldi + c];
}

// At(j, i) = A(i, j) through a 32 x 32 shared-memory tile (padded against bank conflicts):
// reads along A's columns and writes along At's columns are both 128-byte coalesced.
__global__ void transpose_f32_kernel(int64_t m, int64_t n, const float* A, int64_t lda, float* At, int64_t ldt) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  for (int64_t j0 = (int64_t)blockIdx.y * 32; j0 < n; j0 += (int64_t)gridDim.y * 32) {
    for (int c = ty; c < 32; c += 8) {
      const int64_t i = i0 + tx, j = j0 + c;
      if (i < m && j < n) tile[c][tx] = A[j * lda + i];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = i0 + r, j = j0 + tx;
      if (i < m && j < n) At[i * ldt + j] = tile[tx][r];
    }
    __syncthreads();
  }
}

__global__ void fill_kernel(double* d, int64_t count, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = v;
}

}  // namespace

int64_t gemm_num_blocks(int64_t M, int64_t N) { return ((N + BN - 1) / BN) * ((M + BM - 1) / BM); }

// K-split factor: enough CTAs for two waves, chunks of at least 256 along K (16 when the
// output has fewer tiles than an eighth of the SMs, e.g. an FP64 s x s x s product, whose
// few tiles would otherwise leave most of the machine's FP64 units idle).
static int splitk_factor(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = gemm_num_blocks(M, N);
  const int64_t want = 2 * (int64_t)device_sm_count();
  const int64_t min_chunk = tiles * 8 < device_sm_count() ? 16 : 256;
  if (tiles >= want || K < 2 * min_chunk) return 1;
  int64_t z = (want + tiles - 1) / tiles;
  z = std::min<int64_t>(z, K / min_chunk);
  z = std::min<int64_t>(z, 64);
  return (int)std::max<int64_t>(z, 1);
}

size_t gemm_workspace(int64_t M, int64_t N, int64_t K, bool f64) {
  const int z = splitk_factor(M, N, K);
  return z > 1 ? align_up((size_t)z * M * N * (f64 ? 8 : 4)) : 0;
}

cudaError_t launch_gemm(const GemmArgs& a0, bool f64, GemmLeft left, GemmEpi epi, cudaStream_t st) {
  if (a0.M <= 0 || a0.N <= 0) return cudaSuccess;
  if ((a0.M + BM - 1) / BM > 65535) return cudaErrorInvalidValue;
  GemmArgs a = a0;
  int nz = a.splitk_ws ? splitk_factor(a.M, a.N, a.K) : 1;
  if (nz > 1) {
    const int64_t per = (a.K + nz - 1) / nz;
    a.kchunk = (per + BK - 1) / BK * BK;
    nz = (int)((a.K + a.kchunk - 1) / a.kchunk);
  }
  return f64 ? dispatch_epi<double>(a, nz, left, epi, st) : dispatch_epi<float>(a, nz, left, epi, st);
}

static int64_t syrk_ff_chunk(int32_t s, int64_t n) {
  const int64_t nt = (s + FF_T - 1) / FF_T, pairs = nt * (nt + 1) / 2;
  const int64_t want = 2 * (int64_t)device_sm_count();
  int64_t P = std::max<int64_t>(1, std::min<int64_t>((want + pairs - 1) / pairs, (n + 255) / 256));
  return ((n + P - 1) / P + FF_BK - 1) / FF_BK * FF_BK;
}

size_t syrk_ff_workspace(int32_t s, int64_t n) {
  const int64_t P = (n + syrk_ff_chunk(s, n) - 1) / syrk_ff_chunk(s, n);
  return align_up(sizeof(double) * (size_t)P * s * s);
}

cudaError_t launch_syrk_ff(int32_t s, int64_t n, const float* R, int64_t ldr, double* H, int64_t ldh, void* ws,
                           cudaStream_t st) {
  const int64_t nt = (s + FF_T - 1) / FF_T, pairs = nt * (nt + 1) / 2;
  const int64_t chunk = syrk_ff_chunk(s, n);
  const int P = (int)((n + chunk - 1) / chunk);
  double* part = static_cast<double*>(ws);
  {
    KernelTimer kt("gemm_eta_h", st);
    syrk_ff_kernel<<<dim3((unsigned)pairs, (unsigned)P), 256, 0, st>>>(s, n, R, ldr, chunk, part);
  }
  syrk_ff_reduce_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * s + 255) / 256, 1024), 256, 0, st>>>(s, P, part,
                                                                                                          H, ldh);
  note_launches(2);
  return cudaGetLastError();
}

static int gemm_tn_ff_chunks(int32_t s, int64_t n, int64_t m) {
  const int64_t tiles = ((s + FF_T - 1) / FF_T) * ((n + FF_T - 1) / FF_T);
  const int64_t want = 2 * (int64_t)device_sm_count();
  int64_t P = tiles >= want ? 1 : (want + tiles - 1) / tiles;
  P = std::min<int64_t>(P, std::max<int64_t>(1, m / 256));
  return (int)std::min<int64_t>(P, 64);
}

size_t gemm_tn_ff_workspace(int64_t m, int64_t n, int32_t s) {
  const int P = gemm_tn_ff_chunks(s, n, m);
  return P > 1 ? align_up(sizeof(double) * (size_t)P * s * n) : 0;
}

cudaError_t launch_gemm_tn_ff(int64_t m, int64_t n, int32_t s, const float* C, int64_t ldc, const float* B,
                              int64_t ldb, double* out, int64_t ldo, void* ws, const char* timer, cudaStream_t st) {
  if (s <= 0 || n <= 0) return cudaSuccess;
  const int P = gemm_tn_ff_chunks(s, n, m);
  const int64_t chunk = ((m + P - 1) / P + FF_BK - 1) / FF_BK * FF_BK;
  const int Pz = (int)((m + chunk - 1) / chunk);
  const int64_t gx = (n + FF_T - 1) / FF_T;
  if (gx > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)gx, (unsigned)((s + FF_T - 1) / FF_T), (unsigned)std::max(Pz, 1));
  double* dst = Pz > 1 ? static_cast<double*>(ws) : out;
  {
    KernelTimer kt(timer ? timer : "gemm_simt", st);
    gemm_tn_ff_kernel<<<grid, 256, 0, st>>>(s, n, m, C, ldc, B, ldb, chunk, dst, Pz > 1 ? n : ldo, (int64_t)s * n);
  }
  note_launches(1);
  if (Pz > 1) {
    ff_reduce_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * n + 255) / 256, 4096), 256, 0, st>>>(
        s, n, Pz, static_cast<const double*>(ws), out, ldo);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_unit_columns(int32_t s, const int32_t* Js, double* Z, int64_t ldz, cudaStream_t st) {
  unit_columns_kernel<<<(unsigned)std::min<int64_t>(((int64_t)s * s + 255) / 256, 1024), 256, 0, st>>>(s, Js, Z, ldz);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_reduce_sum(const double* partials, int64_t count, double* out, int take_sqrt,
                              cudaStream_t st) {
  reduce_sum_kernel<<<1, 1024, 0, st>>>(partials, count, out, take_sqrt);
  note_launches(1);
  return cudaGetLastError();
}

int64_t sqnorm_num_blocks(int64_t m, int64_t n) { return (n + SQ_COLS - 1) / SQ_COLS; }

cudaError_t launch_sqnorm(int64_t m, int64_t n, skel_dtype dt, const void* A, int64_t lda,
                          double* partials, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (dt == SKEL_F64)
    sqnorm_kernel<double><<<(unsigned)sqnorm_num_blocks(m, n), 256, 0, st>>>(m, n, (const double*)A, lda, partials);
  else
    sqnorm_kernel<float><<<(unsigned)sqnorm_num_blocks(m, n), 256, 0, st>>>(m, n, (const float*)A, lda, partials);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(int64_t m, int32_t s, skel_dtype dt, const void* A, int64_t lda, int64_t ncols,
                               const int32_t* idx, void* C, int64_t ldc, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>((m + 255) / 256, 64), (unsigned)s);
  if (dt == SKEL_F64)
    gather_cols_kernel<double><<<grid, 256, 0, st>>>(m, (const double*)A, lda, ncols, idx, (double*)C, ldc);
  else
    gather_cols_kernel<float><<<grid, 256, 0, st>>>(m, (const float*)A, lda, ncols, idx, (float*)C, ldc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_t(int64_t n, int32_t s, skel_dtype dt, const void* A, int64_t lda, int64_t nrows,
                                 const int32_t* idx, void* Rt, int64_t ldr, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)s);
  if (dt == SKEL_F64)
    gather_rows_t_kernel<double><<<grid, 256, 0, st>>>(n, s, (const double*)A, lda, nrows, idx, (double*)Rt, ldr);
  else
    gather_rows_t_kernel<float><<<grid, 256, 0, st>>>(n, s, (const float*)A, lda, nrows, idx, (float*)Rt, ldr);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols_rowmajor_f64(int32_t s, skel_dtype dt, const void* F, int64_t ldf, int64_t ncols,
                                            const int32_t* idx, double* out, int64_t ldo,
                                            cudaStream_t st) {
  gather_cols_rm_kernel<<<s, 256, 0, st>>>(s, dt, F, ldf, ncols, idx, out, ldo);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_transpose_f64(int32_t s, const double* in, int64_t ldi, double* out,
                                 int64_t ldo, cudaStream_t st) {
  transpose_kernel<<<s, 256, 0, st>>>(s, in, ldi, out, ldo);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_transpose_f32(int64_t m, int64_t n, const float* A, int64_t lda, float* At, int64_t ldt,
                                 cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int64_t gx = (m + 31) / 32;
  if (gx > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)gx, (unsigned)std::min<int64_t>((n + 31) / 32, 65535));
  {
    KernelTimer kt("transpose", st);
    transpose_f32_kernel<<<grid, dim3(32, 8), 0, st>>>(m, n, A, lda, At, ldt);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill_f64(double* d, int64_t count, double value, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  fill_kernel<<<(unsigned)std::min<int64_t>((count + 255) / 256, 1024), 256, 0, st>>>(d, count, value);
  note_launches(1);
  return cudaGetLastError();
}

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace skel
