// Tensor-core Gaussian sketch X = Gamma A (Algorithm 2 line 2; Table 1, T_s = O(nnz(A) l)) on
// sm_103a: tcgen05.mma with FP32 accumulators in tensor memory, A streamed by TMA, Gamma
// generated in shared memory by Philox-4x32-10 + Box-Muller and never written to global
// memory.
//
// Orientation: one CTA computes a 128-row block of X (MMA M = 128 rows of Gamma) for up to
// 512 columns of A (two N = 256 MMAs, 512 TMEM columns), over a K-range of rows of A.
//   MMA A operand = Gamma tile (128 x 32 FP32/TF32), K-major, 128-byte swizzle, generated;
//   MMA B operand = A tile (32 rows of A x 512 columns), K-major (A is column-major),
//                   128-byte swizzle, loaded by TMA exactly as it sits in global memory.
// One generated Gamma tile feeds 512 columns of A (0.25 normals per element of A).  CTAs
// that share the same A tile for different 128-row blocks of X are launched adjacently so
// that the tile is read from HBM once and served from L2 to the others.  A K-split fills
// the machine; partial sums go to a workspace and a reduce kernel applies 1/sqrt(l).
//
// Warp roles (384 threads): warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM allocator,
// warps 4..11 Gamma generators; warps 4..7 then drain TMEM (warp w owns TMEM lanes
// 32*(w%4) .. +31).  Every mbarrier wait is bounded; on timeout the CTA records
// SKEL_ERR_TIMEOUT, stops issuing work, waits (bounded) for what is in flight, frees TMEM
// and returns.
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace skel {

namespace {

using namespace tc;

constexpr int TC_M = 128;
constexpr int TC_BK = 32;             // FP32 elements per 128-byte swizzle row
constexpr int TC_N = 512;             // columns of A per CTA (TMEM columns)
constexpr int TC_ASTAGES = 3;          // TMA stages of A (latency hiding)
constexpr int TC_GSTAGES = 2;          // generated Gamma stages
constexpr int TC_THREADS = 384;
constexpr int TC_GEN_WARP0 = 4;
constexpr int TC_GEN_WARPS = 8;
constexpr uint32_t G_BYTES = TC_M * 128;        // 16 KB per stage
constexpr uint32_t A_BYTES = TC_N * 128;        // 64 KB per stage
constexpr size_t TC_SMEM = 1024 + TC_GSTAGES * G_BYTES + TC_ASTAGES * A_BYTES + 256;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

struct TcParams {
  int64_t m, n;
  int l;
  int64_t k_chunk;        // rows of A per K-split (multiple of TC_BK)
  uint32_t k0s, k1s;      // Philox key
  float* out;             // X (P == 1) or partial buffers [P][l][n]
  int64_t ldo;
  int64_t part_stride;    // elements between partial buffers
  float scale;            // applied when P == 1
  int direct;             // P == 1
  int32_t* dev_status;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
sketch_tc_tf32_kernel(const __grid_constant__ CUtensorMap tmapA, const TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* gbuf = smem;                                  // [GS][G_BYTES]
  unsigned char* abuf = smem + TC_GSTAGES * G_BYTES;           // [AS][A_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(abuf + TC_ASTAGES * A_BYTES);
  // bars: full_a[AS], empty_a[AS], full_g[GS], empty_g[GS], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_ASTAGES + 2 * TC_GSTAGES + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lb = blockIdx.x;                         // 128-row block of X
  const int64_t j0 = (int64_t)blockIdx.y * TC_N;     // first column of A
  const int64_t kb = (int64_t)blockIdx.z * p.k_chunk;
  const int64_t ke = std::min<int64_t>(p.m, kb + p.k_chunk);
  const int nk = (int)((ke - kb + TC_BK - 1) / TC_BK);

  auto full_a = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_a = [&](int s) { return smem_u32(&bars[TC_ASTAGES + s]); };
  auto full_g = [&](int s) { return smem_u32(&bars[2 * TC_ASTAGES + s]); };
  auto empty_g = [&](int s) { return smem_u32(&bars[2 * TC_ASTAGES + TC_GSTAGES + s]); };
  const uint32_t done = smem_u32(&bars[2 * TC_ASTAGES + 2 * TC_GSTAGES]);

  if (tid == 0) {
    for (int s = 0; s < TC_ASTAGES; ++s) {
      mbar_init(full_a(s), 1);
      mbar_init(empty_a(s), 1);
    }
    for (int s = 0; s < TC_GSTAGES; ++s) {
      mbar_init(full_g(s), TC_GEN_WARPS);
      mbar_init(empty_g(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"((uint32_t)TC_N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    if (atomicExch(abort_flag, 1) == 0) record_error(p.dev_status, SKEL_ERR_TIMEOUT, -2);
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % TC_ASTAGES;
        const uint32_t ph = (uint32_t)(it / TC_ASTAGES) & 1u;
        if (*(volatile int*)abort_flag) break;
        if (it >= TC_ASTAGES && !mbar_wait(empty_a(s), ph ^ 1u, TC_WAIT_NS)) { fail(); break; }
        mbar_expect_tx(full_a(s), A_BYTES);
        const int x = (int)(kb + (int64_t)it * TC_BK);
        const uint32_t dst = smem_u32(abuf + s * A_BYTES);
        tma_load_2d(dst, &tmapA, x, (int)j0, full_a(s));
        tma_load_2d(dst + A_BYTES / 2, &tmapA, x, (int)(j0 + TC_N / 2), full_a(s));
        ++issued;
      }
      // drain: every issued load must have landed before the CTA may exit
      for (int it = std::max(0, issued - TC_ASTAGES); it < issued; ++it) {
        const int s = it % TC_ASTAGES;
        if (!mbar_wait(full_a(s), (uint32_t)(it / TC_ASTAGES) & 1u, TC_WAIT_NS)) fail();
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(TC_M, TC_N / 2);
      for (int it = 0; it < nk; ++it) {
        const int sa = it % TC_ASTAGES, sg = it % TC_GSTAGES;
        const uint32_t pa = (uint32_t)(it / TC_ASTAGES) & 1u, pg = (uint32_t)(it / TC_GSTAGES) & 1u;
        if (*(volatile int*)abort_flag) break;
        if (!mbar_wait(full_a(sa), pa, TC_WAIT_NS) || !mbar_wait(full_g(sg), pg, TC_WAIT_NS)) { fail(); break; }
        tc_fence_after();
        const uint32_t ga = smem_u32(gbuf + sg * G_BYTES);
        const uint32_t aa = smem_u32(abuf + sa * A_BYTES);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 8; ++kk) {
          const uint64_t adesc = sw128_desc(ga + kk * 32);
          const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(tmem, adesc, sw128_desc(aa + kk * 32), idesc, acc);
          mma_tf32(tmem + TC_N / 2, adesc, sw128_desc(aa + A_BYTES / 2 + kk * 32), idesc, acc);
        }
        mma_commit(empty_a(sa));
        mma_commit(empty_g(sg));
      }
      mma_commit(done);
    }
  } else if (warp >= TC_GEN_WARP0) {
    // ---------------- Gamma generators ----------------
    const int gt = tid - TC_GEN_WARP0 * 32;            // 0..255
    for (int it = 0; it < nk; ++it) {
      const int s = it % TC_GSTAGES;
      const uint32_t ph = (uint32_t)(it / TC_GSTAGES) & 1u;
      if (*(volatile int*)abort_flag) break;
      if (it >= TC_GSTAGES && !mbar_wait(empty_g(s), ph ^ 1u, TC_WAIT_NS)) { fail(); break; }
      unsigned char* g = gbuf + s * G_BYTES;
      const int64_t kt = kb + (int64_t)it * TC_BK;
#pragma unroll
      for (int q = 0; q < (TC_M * TC_BK / 4) / 256; ++q) {
        const int c = gt + 256 * q;                    // Philox call index in the tile
        const int i = c >> 3, grp = c & 7;             // row of Gamma, 4-column group
        const int64_t row = (int64_t)lb * TC_M + i;
        const int64_t k = kt + 4 * grp;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < p.l && k < p.m) {
          v = gaussian4_f32(p.k0s, p.k1s, (uint32_t)row, (uint32_t)(k >> 2));
          v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w);
          if (k + 1 >= p.m) v.y = 0.f;
          if (k + 2 >= p.m) v.z = 0.f;
          if (k + 3 >= p.m) v.w = 0.f;
        }
        const uint32_t off = (uint32_t)((i >> 3) * 1024 + (i & 7) * 128 + ((grp ^ (i & 7)) << 4));
        *reinterpret_cast<float4*>(g + off) = v;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(full_g(s));
    }
  }

  // ---------------- epilogue: TMEM -> X (warps 4..7) ----------------
  if (warp >= TC_GEN_WARP0 && warp < TC_GEN_WARP0 + 4) {
    const bool ok = mbar_wait(done, 0, TC_WAIT_NS);
    if (!ok) fail();
    tc_fence_after();
    if (ok && !*(volatile int*)abort_flag) {
      const int qd = warp & 3;
      const int64_t row = (int64_t)lb * TC_M + qd * 32 + lane;
      float* orow = p.out + (p.direct ? 0 : (int64_t)blockIdx.z * p.part_stride) + row * p.ldo;
      bool bad = false;
      for (int c0 = 0; c0 < TC_N; c0 += 32) {
        uint32_t r[32];
        TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int64_t jc = j0 + c0;
        if (row < p.l && jc < p.n) {
          const float sc = p.direct ? p.scale : 1.0f;
          if (jc + 32 <= p.n && ((p.ldo & 3) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
              float4 v = make_float4(__uint_as_float(r[q]) * sc, __uint_as_float(r[q + 1]) * sc,
                                     __uint_as_float(r[q + 2]) * sc, __uint_as_float(r[q + 3]) * sc);
              bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
              *reinterpret_cast<float4*>(orow + jc + q) = v;
            }
          } else {
            for (int q = 0; q < 32 && jc + q < p.n; ++q) {
              const float v = __uint_as_float(r[q]) * sc;
              bad |= !isfinite(v);
              orow[jc + q] = v;
            }
          }
        }
      }
      if (bad && p.direct) record_error(p.dev_status, SKEL_ERR_NONFINITE, -1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_N) : "memory");
  }
}

// X = scale * sum_p part[p]; flags non-finite results.
__global__ void tc_reduce_kernel(const float* part, int P, int64_t pstride, int l, int64_t n,
                                 float* X, int64_t ldx, float scale, int32_t* dev_status) {
  bool bad = false;
  for (int r = blockIdx.y; r < l; r += gridDim.y)
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
      const int64_t e = (int64_t)r * n + c;
      float acc = 0.f;
      for (int q = 0; q < P; ++q) acc += part[q * pstride + e];
      const float v = acc * scale;
      bad |= !isfinite(v);
      X[(int64_t)r * ldx + c] = v;
    }
  if (bad) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
}

struct TcPlan {
  int lblocks, jtiles, P;
  int64_t k_chunk;
};

TcPlan plan_tc(int64_t m, int64_t n, int l) {
  TcPlan pl{};
  pl.lblocks = (l + TC_M - 1) / TC_M;
  pl.jtiles = (int)((n + TC_N - 1) / TC_N);
  const int sms = device_sm_count();
  const int64_t ksteps = (m + TC_BK - 1) / TC_BK;
  int P = std::max(1, sms / std::max(1, pl.lblocks * pl.jtiles));
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, ksteps / 8));   // keep >= 8 K-steps per CTA
  pl.P = std::min(P, 16);
  const int64_t steps_per = (ksteps + pl.P - 1) / pl.P;
  pl.k_chunk = steps_per * TC_BK;
  pl.P = (int)((m + pl.k_chunk - 1) / pl.k_chunk);
  return pl;
}

}  // namespace

size_t sketch_tc_workspace(int64_t m, int64_t n, int32_t l) {
  const TcPlan pl = plan_tc(m, n, l);
  return pl.P > 1 ? align_up(sizeof(float) * (size_t)pl.P * l * n) : 0;
}

cudaError_t launch_sketch_tc(int64_t m, int64_t n, const float* A, int64_t lda, int32_t l,
                             skel_prec prec, uint64_t seed, float* X, int64_t ldx, void* ws,
                             int32_t* dev_status, cudaStream_t st) {
  if (prec != SKEL_PREC_TF32) return cudaErrorNotSupported;
  if (m < 1 || n < 1) return cudaErrorNotSupported;
  if ((lda % 4) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
  if (m > (int64_t)INT32_MAX || n > (int64_t)INT32_MAX) return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)n};
  const cuuint64_t gstride[1] = {(cuuint64_t)lda * sizeof(float)};
  const cuuint32_t box[2] = {TC_BK, TC_N / 2};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const TcPlan pl = plan_tc(m, n, l);
  TcParams p{};
  p.m = m; p.n = n; p.l = l;
  p.k_chunk = pl.k_chunk;
  p.k0s = (uint32_t)(seed & 0xffffffffu);
  p.k1s = (uint32_t)(seed >> 32);
  p.direct = pl.P == 1;
  p.scale = (float)(1.0 / std::sqrt((double)l));
  p.out = p.direct ? X : static_cast<float*>(ws);
  p.ldo = p.direct ? ldx : n;
  p.part_stride = (int64_t)l * n;
  p.dev_status = dev_status;
  cudaError_t e = cudaFuncSetAttribute(sketch_tc_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(pl.lblocks, pl.jtiles, pl.P);
  {
    KernelTimer kt("sketch_tc", st);
    sketch_tc_tf32_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(tmap, p);
  }
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || p.direct) return e;
  tc_reduce_kernel<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(l, 128)), 256, 0, st>>>(
      static_cast<const float*>(ws), pl.P, p.part_stride, l, n, X, ldx, p.scale, dev_status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
