// Rank-b update C += alpha A B for FP32, with a short inner dimension (b <= 64): the trailing
// updates of the panel-blocked Householder QR (C(t0:, t0+b:) -= (V_p T_p^T) W) and the
// formation of Q_C (E(t0:, :) -= (V_p T_p) Y), Remark 3 / Eq. (2.1).  A is column-major
// (M x K), B row-major (K x N), C column-major (M x N).
//
// The work is bound by reading and writing C once (2 K flops per 8 bytes of C): one CTA takes
// a 128 x 128 tile of C, stages all K columns of A's tile and K rows of B's tile in shared
// memory (float4 loads where the operands are 16-byte aligned), and every thread accumulates an
// 8 x 8 block in registers (64 FFMA per four 16-byte shared loads), then reads its block of C,
// adds, and writes it back (each warp touching 512 contiguous bytes per column).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int RU_M = 128, RU_N = 128, RU_KMAX = 64, RU_THREADS = 256;
constexpr size_t RU_SMEM = sizeof(float) * (size_t)RU_KMAX * (RU_M + RU_N);

struct RankUpdateArgs {
  int64_t M, N;
  int K;
  const float* A; int64_t lda;
  const float* B; int64_t ldb;
  float* C; int64_t ldc;
  float alpha;
  bool vec_a, vec_b, vec_c;    // 16-byte aligned rows (A, C) / columns (B) of the tiles
};

__global__ void __launch_bounds__(RU_THREADS, 2) rank_update_kernel(const RankUpdateArgs a) {
  extern __shared__ __align__(16) float ru_smem[];
  float* As = ru_smem;                       // [K][RU_M]: As[k][r] = A(r0 + r, k)
  float* Bs = ru_smem + RU_KMAX * RU_M;      // [K][RU_N]: Bs[k][c] = B(k, c0 + c)
  const int tid = threadIdx.x;
  const int ty = tid & 15, tx = tid >> 4;    // rows ty*8 .. +7, columns tx*8 .. +7
  const int64_t r0 = (int64_t)blockIdx.x * RU_M, c0 = (int64_t)blockIdx.y * RU_N;
  const int K = a.K;

  // stage A's and B's tiles: RU_M / 4 (RU_N / 4) groups of four per row of K
  for (int e = tid; e < K * (RU_M / 4); e += RU_THREADS) {
    const int k = e / (RU_M / 4), r = 4 * (e % (RU_M / 4));
    const int64_t gr = r0 + r;
    float4 v;
    if (a.vec_a && gr + 3 < a.M) {
      v = __ldg(reinterpret_cast<const float4*>(a.A + gr + (int64_t)k * a.lda));
    } else {
      const float* p = a.A + (int64_t)k * a.lda;
      v.x = gr < a.M ? __ldg(p + gr) : 0.f;
      v.y = gr + 1 < a.M ? __ldg(p + gr + 1) : 0.f;
      v.z = gr + 2 < a.M ? __ldg(p + gr + 2) : 0.f;
      v.w = gr + 3 < a.M ? __ldg(p + gr + 3) : 0.f;
    }
    *reinterpret_cast<float4*>(As + k * RU_M + r) = v;
  }
  for (int e = tid; e < K * (RU_N / 4); e += RU_THREADS) {
    const int k = e / (RU_N / 4), c = 4 * (e % (RU_N / 4));
    const int64_t gc = c0 + c;
    float4 v;
    const float* p = a.B + (int64_t)k * a.ldb;
    if (a.vec_b && gc + 3 < a.N) {
      v = __ldg(reinterpret_cast<const float4*>(p + gc));
    } else {
      v.x = gc < a.N ? __ldg(p + gc) : 0.f;
      v.y = gc + 1 < a.N ? __ldg(p + gc + 1) : 0.f;
      v.z = gc + 2 < a.N ? __ldg(p + gc + 2) : 0.f;
      v.w = gc + 3 < a.N ? __ldg(p + gc + 3) : 0.f;
    }
    *reinterpret_cast<float4*>(Bs + k * RU_N + c) = v;
  }
  __syncthreads();

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + k * RU_M + ty * 8);
    const float4 a1 = *reinterpret_cast<const float4*>(As + k * RU_M + ty * 8 + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + k * RU_N + tx * 8);
    const float4 b1 = *reinterpret_cast<const float4*>(Bs + k * RU_N + tx * 8 + 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }

  // C(rows, col) += alpha acc, one column of the thread's block at a time
  const int64_t gr = r0 + ty * 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t gc = c0 + tx * 8 + j;
    if (gc >= a.N) break;
    float* p = a.C + gc * a.ldc + gr;
    if (a.vec_c && gr + 7 < a.M) {
      float4 x0 = *reinterpret_cast<const float4*>(p);
      float4 x1 = *reinterpret_cast<const float4*>(p + 4);
      x0.x = fmaf(a.alpha, acc[0][j], x0.x); x0.y = fmaf(a.alpha, acc[1][j], x0.y);
      x0.z = fmaf(a.alpha, acc[2][j], x0.z); x0.w = fmaf(a.alpha, acc[3][j], x0.w);
      x1.x = fmaf(a.alpha, acc[4][j], x1.x); x1.y = fmaf(a.alpha, acc[5][j], x1.y);
      x1.z = fmaf(a.alpha, acc[6][j], x1.z); x1.w = fmaf(a.alpha, acc[7][j], x1.w);
      *reinterpret_cast<float4*>(p) = x0;
      *reinterpret_cast<float4*>(p + 4) = x1;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (gr + i < a.M) p[i] = fmaf(a.alpha, acc[i][j], p[i]);
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_rank_update_f32(int64_t M, int64_t N, int K, const float* A, int64_t lda, const float* B,
                                   int64_t ldb, float* C, int64_t ldc, float alpha, const char* timer,
                                   cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (K > RU_KMAX || lda < M || ldb < N || ldc < M) return cudaErrorInvalidValue;
  const int64_t gx = (M + RU_M - 1) / RU_M, gy = (N + RU_N - 1) / RU_N;
  if (gx > (int64_t)INT32_MAX || gy > 65535) return cudaErrorInvalidValue;
  const cudaError_t e = cudaFuncSetAttribute(rank_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RU_SMEM);
  if (e != cudaSuccess) return e;
  RankUpdateArgs a{M, N, K, A, lda, B, ldb, C, ldc, alpha,
                   aligned16(A) && lda % 4 == 0, aligned16(B) && ldb % 4 == 0, aligned16(C) && ldc % 4 == 0};
  {
    KernelTimer kt(timer ? timer : "gemm_simt", st);
    rank_update_kernel<<<dim3((unsigned)gx, (unsigned)gy), RU_THREADS, RU_SMEM, st>>>(a);
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
