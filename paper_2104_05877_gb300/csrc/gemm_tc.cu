// W = Q^T A on the tensor cores with FP32-level accuracy (3xTF32), for the column ID
// Z = R_C^{-1} Q_C^T A (Eq. (2.1)), the stable CUR (Remark 3) and the Gram-identity error
// ||A||^2 - ||Q_C^T A||^2.  Q (m x s) and A (m x n) are FP32, column-major; W is s x n
// row-major FP32.
//
// Every operand is split into two TF32 numbers, x = hi(x) + lo(x) with hi = rn_tf32(x) and
// lo = rn_tf32(x - hi), and W = Qhi^T Ahi + (Qhi^T Alo + Qlo^T Ahi) is accumulated in FP32 in
// tensor memory, the main product and the two corrections in separate accumulators that the
// epilogue adds (the dropped Qlo^T Alo term is below FP32 rounding).  The accumulation inside
// the tensor core is not correctly rounded, so its error grows with the number of MMAs per
// accumulator: a CTA covers at most kGtKChunk rows of K and the K-split partials are summed in
// FP64.  Both halves are rounded
// explicitly, so the products are exact in whatever way the tensor core reads TF32.  Qhi and
// Qlo are prepared once per call (Q is small); the tile of A is split in shared memory as it
// arrives.
//
// Orientation (as the sketch kernel): one CTA computes 128 rows of W for 256 columns of A over
// a K-range of rows of A.  Per 32-row step of K:
//   TMA: A tile (32 x 256, K-major, 128-byte swizzle), Qhi and Qlo tiles (128 x 32).
//   8 converter warps: A tile -> Ahi in place, Alo beside it (positions are preserved, so the
//     swizzle does not matter).
//   MMA warp: 4 x 3 tcgen05.mma kind::tf32 (M 128, N 256, K 8) into one accumulator.
// Two stages; every mbarrier wait is bounded (SKEL_ERR_TIMEOUT, then drain and free TMEM).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace skel {

namespace {

using namespace tc;

constexpr int GT_M = 128;
constexpr int GT_BK = 32;
constexpr int GT_N = 256;
constexpr int GT_STAGES = 2;
constexpr int GT_THREADS = 384;
constexpr int GT_CONV_WARP0 = 4;
constexpr int GT_CONV_WARPS = 8;
constexpr uint32_t GT_A_BYTES = GT_N * 128;     // 32 KB
constexpr uint32_t GT_Q_BYTES = GT_M * 128;     // 16 KB
constexpr uint32_t GT_STAGE_BYTES = 2 * GT_A_BYTES + 2 * GT_Q_BYTES;
constexpr size_t GT_SMEM = 1024 + GT_STAGES * GT_STAGE_BYTES + 256;
constexpr uint64_t GT_WAIT_NS = 2000000000ull;
constexpr int64_t kGtKChunk = 1024;             // rows of K per CTA (accumulation depth)

struct GtParams {
  int64_t m, n;
  int s;
  int64_t k_chunk;        // rows of A per K-split (multiple of GT_BK)
  float* out;             // W (direct) or partial buffers [P][s][n]
  int64_t ldo;
  int64_t part_stride;
  int direct;
  double* sq_partials;    // direct and non-null: one partial sum of squares per CTA
  int32_t* dev_status;
};

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(GT_THREADS, 1)
gemm_tn_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQhi,
                      const __grid_constant__ CUtensorMap tmQlo, const GtParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s: [A/Ahi 32 KB][Alo 32 KB][Qhi 16 KB][Qlo 16 KB]
  auto a_buf = [&](int s) { return smem + s * GT_STAGE_BYTES; };
  auto alo_buf = [&](int s) { return smem + s * GT_STAGE_BYTES + GT_A_BYTES; };
  auto qhi_buf = [&](int s) { return smem + s * GT_STAGE_BYTES + 2 * GT_A_BYTES; };
  auto qlo_buf = [&](int s) { return smem + s * GT_STAGE_BYTES + 2 * GT_A_BYTES + GT_Q_BYTES; };
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + GT_STAGES * GT_STAGE_BYTES);
  // bars: full[S], conv[S], empty[S], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * GT_STAGES + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  float* red = reinterpret_cast<float*>(abort_flag + 1);     // 4 warp partials (epilogue)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mb = blockIdx.x;                          // 128-row block of W
  const int64_t j0 = (int64_t)blockIdx.y * GT_N;      // first column of A
  const int64_t kb = (int64_t)blockIdx.z * p.k_chunk;
  const int64_t ke = std::min<int64_t>(p.m, kb + p.k_chunk);
  const int nk = (int)((ke - kb + GT_BK - 1) / GT_BK);

  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto conv = [&](int s) { return smem_u32(&bars[GT_STAGES + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * GT_STAGES + s]); };
  const uint32_t done = smem_u32(&bars[3 * GT_STAGES]);

  if (tid == 0) {
    for (int s = 0; s < GT_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), GT_CONV_WARPS);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"((uint32_t)(2 * GT_N)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    if (atomicExch(abort_flag, 1) == 0) record_error(p.dev_status, SKEL_ERR_TIMEOUT, -3);
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % GT_STAGES;
        const uint32_t ph = (uint32_t)(it / GT_STAGES) & 1u;
        if (*(volatile int*)abort_flag) break;
        if (it >= GT_STAGES && !mbar_wait(empty(s), ph ^ 1u, GT_WAIT_NS)) { fail(); break; }
        mbar_expect_tx(full(s), GT_A_BYTES + 2 * GT_Q_BYTES);
        const int x = (int)(kb + (int64_t)it * GT_BK);
        tma_load_2d(smem_u32(a_buf(s)), &tmA, x, (int)j0, full(s));
        tma_load_2d(smem_u32(qhi_buf(s)), &tmQhi, x, mb * GT_M, full(s));
        tma_load_2d(smem_u32(qlo_buf(s)), &tmQlo, x, mb * GT_M, full(s));
        ++issued;
      }
      // drain: every issued load must have landed before the CTA may exit
      for (int it = std::max(0, issued - GT_STAGES); it < issued; ++it) {
        const int s = it % GT_STAGES;
        if (!mbar_wait(full(s), (uint32_t)(it / GT_STAGES) & 1u, GT_WAIT_NS)) fail();
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(GT_M, GT_N);
      for (int it = 0; it < nk; ++it) {
        const int s = it % GT_STAGES;
        const uint32_t ph = (uint32_t)(it / GT_STAGES) & 1u;
        if (*(volatile int*)abort_flag) break;
        if (!mbar_wait(conv(s), ph, GT_WAIT_NS)) { fail(); break; }
        tc_fence_after();
        const uint32_t ahi = smem_u32(a_buf(s)), alo = smem_u32(alo_buf(s));
        const uint32_t qhi = smem_u32(qhi_buf(s)), qlo = smem_u32(qlo_buf(s));
#pragma unroll
        for (int kk = 0; kk < GT_BK / 8; ++kk) {
          const uint32_t acc0 = (it > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(tmem, sw128_desc(qhi + kk * 32), sw128_desc(ahi + kk * 32), idesc, acc0);
          mma_tf32(tmem + GT_N, sw128_desc(qlo + kk * 32), sw128_desc(ahi + kk * 32), idesc, acc0);
          mma_tf32(tmem + GT_N, sw128_desc(qhi + kk * 32), sw128_desc(alo + kk * 32), idesc, 1u);
        }
        mma_commit(empty(s));
      }
      mma_commit(done);
    }
  } else if (warp >= GT_CONV_WARP0) {
    // ---------------- converters: A -> Ahi (in place), Alo ----------------
    const int ct = tid - GT_CONV_WARP0 * 32;             // 0..255
    for (int it = 0; it < nk; ++it) {
      const int s = it % GT_STAGES;
      const uint32_t ph = (uint32_t)(it / GT_STAGES) & 1u;
      if (*(volatile int*)abort_flag) break;
      if (!mbar_wait(full(s), ph, GT_WAIT_NS)) { fail(); break; }
      float4* a = reinterpret_cast<float4*>(a_buf(s));
      float4* lo = reinterpret_cast<float4*>(alo_buf(s));
#pragma unroll
      for (int q = 0; q < (int)(GT_A_BYTES / 16) / 256; ++q) {
        const int e = ct + 256 * q;
        const float4 v = a[e];
        float4 h, l;
        h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
        h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
        h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
        h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
        a[e] = h;
        lo[e] = l;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(conv(s));
    }
  }

  // ---------------- epilogue: TMEM -> W (warps 4..7) ----------------
  double sq = 0.0;
  if (warp >= GT_CONV_WARP0 && warp < GT_CONV_WARP0 + 4) {
    const bool ok = mbar_wait(done, 0, GT_WAIT_NS);
    if (!ok) fail();
    tc_fence_after();
    if (ok && !*(volatile int*)abort_flag) {
      const int qd = warp & 3;
      const int64_t row = (int64_t)mb * GT_M + qd * 32 + lane;
      float* orow = p.out + (p.direct ? 0 : (int64_t)blockIdx.z * p.part_stride) + row * p.ldo;
      for (int c0 = 0; c0 < GT_N; c0 += 32) {
        uint32_t r[32], rc[32];
        TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r);
        TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(GT_N + c0), rc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 32; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) + __uint_as_float(rc[q]));
        const int64_t jc = j0 + c0;
        if (row < p.s && jc < p.n) {
          if (jc + 32 <= p.n && ((p.ldo & 3) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
              const float4 v = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                                           __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
              sq += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
              *reinterpret_cast<float4*>(orow + jc + q) = v;
            }
          } else {
            for (int q = 0; q < 32 && jc + q < p.n; ++q) {
              const float v = __uint_as_float(r[q]);
              sq += (double)v * v;
              orow[jc + q] = v;
            }
          }
        }
      }
    }
  }
  if (p.direct && p.sq_partials) {
    // fixed-order sum of the 128 epilogue rows: lanes, then the four warps
    if (warp >= GT_CONV_WARP0 && warp < GT_CONV_WARP0 + 4) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    double* redd = reinterpret_cast<double*>(((uintptr_t)red + 7) & ~(uintptr_t)7);
    if (warp >= GT_CONV_WARP0 && warp < GT_CONV_WARP0 + 4 && lane == 0) redd[warp - GT_CONV_WARP0] = sq;
    __syncthreads();
    if (tid == 0)
      p.sq_partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x)] = redd[0] + redd[1] + redd[2] + redd[3];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * GT_N)) : "memory");
  }
}

// Qhi, Qlo (m x s, leading dimension ldh) from Q.
__global__ void split_tf32_kernel(const float* Q, int64_t ldq, int64_t m, int s, float* hi, float* lo, int64_t ldh) {
  for (int c = blockIdx.y; c < s; c += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
      const float v = Q[i + (int64_t)c * ldq];
      const float h = tf32_rn(v);
      hi[i + (int64_t)c * ldh] = h;
      lo[i + (int64_t)c * ldh] = tf32_rn(v - h);
    }
}

// leading dimension of the split copies of Q: a multiple of 4 elements (16-byte TMA strides)
int64_t split_ld(int64_t m) { return (m + 3) / 4 * 4; }

// W = sum_p part[p] (in split order); one partial sum of squares per CTA (fixed order) when
// requested.  CTA (x, r): row r, columns 1024x .. 1024x+1023, four per thread.
constexpr int GT_RED_COLS = 1024;
__global__ void __launch_bounds__(256) gt_reduce_kernel(const float* part, int P, int64_t pstride, int s, int64_t n,
                                                        float* W, int64_t ldw, double* sq_partials) {
  const int r = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * GT_RED_COLS + 4 * threadIdx.x;
  double sq = 0.0;
  if (c < n) {
    const float* src = part + (int64_t)r * n + c;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (c + 4 <= n && (n & 3) == 0) {
      int q = 0;
      for (; q + 4 <= P; q += 4) {             // four independent loads in flight
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(src + (q + u) * pstride);
#pragma unroll
        for (int u = 0; u < 4; ++u) { a[0] += v[u].x; a[1] += v[u].y; a[2] += v[u].z; a[3] += v[u].w; }
      }
      for (; q < P; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(src + q * pstride);
        a[0] += v.x; a[1] += v.y; a[2] += v.z; a[3] += v.w;
      }
    } else {
      for (int u = 0; u < 4 && c + u < n; ++u)
        for (int q = 0; q < P; ++q) a[u] += src[q * pstride + u];
    }
    float* dst = W + (int64_t)r * ldw + c;
    for (int u = 0; u < 4 && c + u < n; ++u) {
      dst[u] = a[u];
      sq += (double)a[u] * a[u];
    }
  }
  if (sq_partials) {
    const double tot = block_sum<double>(sq);
    if (threadIdx.x == 0) sq_partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

struct GtPlan {
  int mblocks, jtiles, P;
  int64_t k_chunk;
};

GtPlan plan_gt(int64_t m, int64_t n, int s) {
  GtPlan pl{};
  pl.mblocks = (s + GT_M - 1) / GT_M;
  pl.jtiles = (int)((n + GT_N - 1) / GT_N);
  const int sms = device_sm_count();
  const int64_t ksteps = (m + GT_BK - 1) / GT_BK;
  int P = std::max(1, sms / std::max(1, pl.mblocks * pl.jtiles));
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, ksteps / 8));
  P = (int)std::max<int64_t>(P, (m + kGtKChunk - 1) / kGtKChunk);
  pl.P = std::min(P, 64);
  const int64_t steps_per = (ksteps + pl.P - 1) / pl.P;
  pl.k_chunk = steps_per * GT_BK;
  pl.P = (int)((m + pl.k_chunk - 1) / pl.k_chunk);
  return pl;
}

}  // namespace

bool gemm_tc_usable(int64_t m, int64_t n, int32_t s, const void* Q, int64_t ldq, const void* A, int64_t lda) {
  if (m < 1 || n < 1 || s < 1 || m > (int64_t)INT32_MAX || n > (int64_t)INT32_MAX) return false;
  if ((lda % 4) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return false;
  (void)Q; (void)ldq;
  return encode_fn() != nullptr;
}

size_t gemm_tc_workspace(int64_t m, int64_t n, int32_t s) {
  const GtPlan pl = plan_gt(m, n, s);
  return 2 * align_up(sizeof(float) * (size_t)split_ld(m) * s) +
         (pl.P > 1 ? align_up(sizeof(float) * (size_t)pl.P * s * n) : 0);
}

size_t gemm_tc_workspace_bound(int64_t m, int64_t nmax, int32_t s) {
  // the K-split never exceeds 64 partial buffers (plan_gt)
  return 2 * align_up(sizeof(float) * (size_t)split_ld(m) * s) + align_up(sizeof(float) * (size_t)64 * s * nmax);
}

int64_t gemm_tc_num_partials(int64_t m, int64_t n, int32_t s) {
  const GtPlan pl = plan_gt(m, n, s);
  return pl.P > 1 ? (int64_t)s * ((n + GT_RED_COLS - 1) / GT_RED_COLS) : (int64_t)pl.mblocks * pl.jtiles;
}

cudaError_t launch_gemm_tc_tn(int64_t m, int64_t n, int32_t s, const float* Q, int64_t ldq, const float* A,
                              int64_t lda, float* W, int64_t ldw, double* sq_partials, void* ws,
                              int32_t* dev_status, cudaStream_t st, const char* timer) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const GtPlan pl = plan_gt(m, n, s);
  const int64_t ldh = split_ld(m);
  char* base = static_cast<char*>(ws);
  float* qhi = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * (size_t)ldh * s);
  float* qlo = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * (size_t)ldh * s);
  float* part = reinterpret_cast<float*>(base);
  split_tf32_kernel<<<dim3((unsigned)std::min<int64_t>((m + 255) / 256, 64), (unsigned)std::min(s, 256)), 256, 0, st>>>(
      Q, ldq, m, s, qhi, qlo, ldh);
  note_launches(1);
  CUtensorMap tA, tQh, tQl;
  const cuuint32_t estride[2] = {1, 1};
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)lda * sizeof(float)};
    const cuuint32_t box[2] = {GT_BK, GT_N};
    if (enc(&tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)s};
    const cuuint64_t gstride[1] = {(cuuint64_t)ldh * sizeof(float)};
    const cuuint32_t box[2] = {GT_BK, GT_M};
    if (enc(&tQh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, qhi, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&tQl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, qlo, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  GtParams p{};
  p.m = m; p.n = n; p.s = s;
  p.k_chunk = pl.k_chunk;
  p.direct = pl.P == 1;
  p.out = p.direct ? W : part;
  p.ldo = p.direct ? ldw : n;
  p.part_stride = (int64_t)s * n;
  p.sq_partials = p.direct ? sq_partials : nullptr;
  p.dev_status = dev_status;
  cudaError_t e = cudaFuncSetAttribute(gemm_tn_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GT_SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(pl.mblocks, pl.jtiles, pl.P);
  {
    KernelTimer kt(timer, st);
    gemm_tn_tf32x3_kernel<<<grid, GT_THREADS, GT_SMEM, st>>>(tA, tQh, tQl, p);
  }
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || p.direct) return e;
  gt_reduce_kernel<<<dim3((unsigned)((n + GT_RED_COLS - 1) / GT_RED_COLS), (unsigned)s), 256, 0, st>>>(
      part, pl.P, p.part_stride, s, n, W, ldw, sq_partials);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
