// FP8 (e4m3) Gaussian sketch X = Gamma A (Algorithm 2, sketch step) on sm_103a tensor cores.
//
// Quantisation: every column of A has one power-of-two scale, s = 2^ceil(log2(amax / 448))
// (the smallest that keeps the column inside e4m3's range), and A8 = e4m3(A / s) rounded to
// nearest even (the division is exact).  The standard normals are rounded to e4m3 unscaled
// (|g| < 448).  Products of two e4m3 numbers are exact in FP32.
//
// Kernels:
//   fp8_quantize_kernel  one CTA per column at a time: amax over the column, the scale, then
//                        the codes (the column's second read is served from L2: few columns
//                        are in flight at once).
//   fp8_gamma_kernel     e4m3 normals G8 (l_pad x m_pad bytes, zero padded), 0.35 l m bytes
//                        that stay in L2.
//   sketch_fp8_kernel    one CTA per 128 rows of X x 512 columns of A over an interleaved
//                        K-split of 128-row blocks: TMA brings the A8 and G8 tiles (128-byte
//                        swizzle, 128 K-elements per row; one G8 tile serves four 128-column
//                        quarters of A8), tcgen05.mma kind::f8f6f4 (M 128, N 256, K 32, two per
//                        K-step) accumulates the CTA's whole K range in 512 TMEM columns,
//                        and four epilogue warps multiply each column by its scale once at
//                        the end (the scale is constant along K).
// Every mbarrier wait is bounded (SKEL_ERR_TIMEOUT, then drain and free TMEM).
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace skel {

namespace {

using namespace tc;

constexpr int F8_BLOCK = 128;                 // rows per scale block = K per stage
constexpr int F8_N = 512;                     // columns of A per CTA: two N = 256 MMAs
constexpr int F8_STAGES = 2;
constexpr int F8_THREADS = 256;               // warp 0 TMA, 1 MMA, 2 TMEM, 4..7 epilogue
constexpr uint32_t F8_GTILE = 128 * 128;                  // G8 tile: 128 rows of Gamma x 128 K bytes
constexpr uint32_t F8_ATILE = F8_N * 128;                 // A8 tile: 512 columns of A x 128 K bytes
constexpr uint32_t F8_STAGE = F8_ATILE + F8_GTILE;        // a multiple of 1024 (128-byte swizzle atoms)
constexpr size_t F8_SMEM = 1024 + F8_STAGES * (size_t)F8_STAGE + 256;
constexpr uint64_t F8_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));   // low byte = a
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

constexpr int kQG = 8;                        // 16-byte loads in flight per quantisation thread

// One CTA per column j (grid-stride): amax by thread, warp and CTA reductions, the scale S[j],
// then the codes, thread t covering rows 4t .. 4t+3 of every 4 * blockDim.x.
__global__ void fp8_quantize_kernel(int64_t m, int64_t n, const float* A, int64_t lda, uint8_t* A8, int64_t ld8,
                                    float* S, int32_t* dev_status) {
  __shared__ uint32_t wmax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto load4 = [&](const float* col, int64_t r, float (&v)[4]) {
    if (r >= m) {
      v[0] = v[1] = v[2] = v[3] = 0.f;
    } else if (r + 3 < m) {
      const float4 q = *reinterpret_cast<const float4*>(col + r);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
      for (int u = 0; u < 4; ++u) v[u] = r + u < m ? col[r + u] : 0.f;
    }
  };
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const float* col = A + j * lda;
    uint32_t bits = 0;
    const int64_t step = 4 * (int64_t)blockDim.x;
    for (int64_t r0 = 4 * (int64_t)threadIdx.x; r0 < m; r0 += kQG * step) {   // kQG loads in flight
      float v[kQG][4];
#pragma unroll
      for (int g = 0; g < kQG; ++g) load4(col, r0 + g * step, v[g]);
#pragma unroll
      for (int g = 0; g < kQG; ++g)
#pragma unroll
        for (int u = 0; u < 4; ++u) bits = max(bits, __float_as_uint(fabsf(v[g][u])));
    }
    bits = __reduce_max_sync(0xffffffffu, bits);
    if (lane == 0) wmax[warp] = bits;
    __syncthreads();
    bits = 0;
    for (int w = 0; w < nw; ++w) bits = max(bits, wmax[w]);
    float scale = 1.f, inv = 1.f;
    if (bits >= 0x7f800000u) {
      if (threadIdx.x == 0) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
    } else if (bits != 0u) {
      // amax = f 2^E, f in [0.5, 1): the smallest e with 448 2^e >= amax is E - 9, or E - 8
      // when f > 0.875 (448 = 0.875 2^9)
      int E;
      const float f = frexpf(__uint_as_float(bits), &E);
      const int e = max(-126, min(127, f > 0.875f ? E - 8 : E - 9));
      scale = ldexpf(1.f, e);
      inv = ldexpf(1.f, -e);
    }
    if (threadIdx.x == 0) S[j] = scale;
    uint8_t* dst = A8 + j * ld8;
    for (int64_t r0 = 4 * (int64_t)threadIdx.x; r0 < m; r0 += kQG * step) {
      float v[kQG][4];
#pragma unroll
      for (int g = 0; g < kQG; ++g) load4(col, r0 + g * step, v[g]);
#pragma unroll
      for (int g = 0; g < kQG; ++g) {
        const int64_t r = r0 + g * step;
        if (r >= m) continue;
        const uint32_t word = e4m3x4(v[g][0] * inv, v[g][1] * inv, v[g][2] * inv, v[g][3] * inv);
        if (r + 3 < m) {
          *reinterpret_cast<uint32_t*>(dst + r) = word;
        } else {
          for (int u = 0; u < 4 && r + u < m; ++u) dst[r + u] = (uint8_t)(word >> (8 * u));
        }
      }
    }
    __syncthreads();                 // wmax is rewritten for the next column
  }
}

// G8 (lp x mg bytes, row-major): e4m3 of the standard normals for i < l, k < m; zero elsewhere.
__global__ void fp8_gamma_kernel(int l, int lp, int64_t m, int64_t mg, uint32_t k0, uint32_t k1, uint8_t* G8) {
  const int64_t m4 = mg / 4;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)lp * m4;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m4);
    const int64_t j4 = e % m4;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < l && 4 * j4 < m) {
      g = gaussian4_f32(k0, k1, (uint32_t)i, (uint32_t)j4);
      if (4 * j4 + 1 >= m) g.y = 0.f;
      if (4 * j4 + 2 >= m) g.z = 0.f;
      if (4 * j4 + 3 >= m) g.w = 0.f;
    }
    reinterpret_cast<uint32_t*>(G8 + (int64_t)i * mg)[j4] = e4m3x4(g.x, g.y, g.z, g.w);
  }
}

// Instruction descriptor for kind::f8f6f4: D FP32, A and B e4m3, both K-major, M x N.
constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

struct F8Params {
  int64_t m, n;
  int l, P;                 // K-split: CTA z takes the row blocks z, z + P, ...
  int64_t nkb;              // 128-row blocks over m
  const float* S;           // column scales [n]
  float* out;               // X (P == 1) or partial buffers [P][l][n]
  int64_t ldo, part_stride;
  float scale;              // 1 / sqrt(l), applied when P == 1
  int direct;
  int32_t* dev_status;
};

__global__ void __launch_bounds__(F8_THREADS, 1)
sketch_fp8_kernel(const __grid_constant__ CUtensorMap tmA8, const __grid_constant__ CUtensorMap tmG8,
                  const F8Params p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + F8_STAGES * F8_STAGE);
  // bars: full[S], empty[S], tfull[2], tempty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * F8_STAGES + 4);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lb = blockIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * F8_N;
  const int kz = blockIdx.z;
  const int nk = (int)((p.nkb - kz + p.P - 1) / p.P);
  auto a_buf = [&](int s) { return smem + s * F8_STAGE; };
  auto g_buf = [&](int s) { return smem + s * F8_STAGE + F8_ATILE; };
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[F8_STAGES + s]); };
  auto tfull = [&](int b) { return smem_u32(&bars[2 * F8_STAGES + b]); };
  auto tempty = [&](int b) { return smem_u32(&bars[2 * F8_STAGES + 2 + b]); };

  if (tid == 0) {
    for (int s = 0; s < F8_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"((uint32_t)F8_N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    if (atomicExch(abort_flag, 1) == 0) record_error(p.dev_status, SKEL_ERR_TIMEOUT, -2);
  };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % F8_STAGES;
        const uint32_t ph = (uint32_t)(it / F8_STAGES) & 1u;
        if (aborted()) break;
        if (it >= F8_STAGES && !mbar_wait(empty(s), ph ^ 1u, F8_WAIT_NS)) { fail(); break; }
        mbar_expect_tx(full(s), F8_STAGE);
        const int x = (int)(((int64_t)kz + (int64_t)it * p.P) * F8_BLOCK);
        tma_load_2d(smem_u32(a_buf(s)), &tmA8, x, (int)j0, full(s));               // columns j0 .. +255
        tma_load_2d(smem_u32(a_buf(s)) + 256 * 128, &tmA8, x, (int)j0 + 256, full(s));   // .. +511
        tma_load_2d(smem_u32(g_buf(s)), &tmG8, x, lb * 128, full(s));
        ++issued;
      }
      for (int it = std::max(0, issued - F8_STAGES); it < issued; ++it)
        if (!mbar_wait(full(it % F8_STAGES), (uint32_t)(it / F8_STAGES) & 1u, F8_WAIT_NS)) fail();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_e4m3(128, 256);
      for (int it = 0; it < nk; ++it) {
        const int s = it % F8_STAGES;
        const uint32_t ph = (uint32_t)(it / F8_STAGES) & 1u;
        if (aborted()) break;
        if (!mbar_wait(full(s), ph, F8_WAIT_NS)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t ga = smem_u32(g_buf(s)), aa = smem_u32(a_buf(s));
#pragma unroll
        for (int kk = 0; kk < F8_BLOCK / 32; ++kk) {    // K = 32 per MMA: 32 bytes of each row
          const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
          mma_f8(tmem, sw128_desc(ga + kk * 32), sw128_desc(aa + kk * 32), idesc, acc);
          mma_f8(tmem + 256, sw128_desc(ga + kk * 32), sw128_desc(aa + 256 * 128 + kk * 32), idesc, acc);
        }
        mma_commit(empty(s));
      }
      mma_commit(tfull(0));      // arrives once every MMA issued above has completed
    }
  } else if (warp >= 4) {
    // epilogue warps: row i of X per thread, read from TMEM once the whole K range is in
    const int qd = warp & 3;
    const int64_t i = (int64_t)lb * 128 + qd * 32 + lane;
    bool ok = true;
    if (nk > 0 && !mbar_wait(tfull(0), 0u, F8_WAIT_NS)) {
      fail();
      ok = false;
    }
    tc_fence_after();
    if (ok && !aborted()) {
      float* orow = p.out + (p.direct ? 0 : (int64_t)kz * p.part_stride) + i * p.ldo;
      const float scl = p.direct ? p.scale : 1.f;
      // 16-byte stores when every row of the output starts on a 16-byte boundary (S is
      // 256-byte aligned in the workspace)
      const bool vec = (p.ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0 &&
                       (p.part_stride & 3) == 0;
      bool bad = false;
      for (int c0 = 0; c0 < F8_N; c0 += 32) {
        uint32_t r[32];
        if (nk > 0) {
          TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) r[q] = 0u;
        }
        if (i < p.l) {
          const int64_t jb = j0 + c0;
          if (jb + 32 <= p.n && vec) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
              const float4 sc = __ldg(reinterpret_cast<const float4*>(p.S + jb + q));
              const float4 v = make_float4(__uint_as_float(r[q]) * sc.x * scl, __uint_as_float(r[q + 1]) * sc.y * scl,
                                           __uint_as_float(r[q + 2]) * sc.z * scl, __uint_as_float(r[q + 3]) * sc.w * scl);
              bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
              *reinterpret_cast<float4*>(orow + jb + q) = v;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              const int64_t jc = jb + q;
              if (jc < p.n) {
                const float v = __uint_as_float(r[q]) * __ldg(p.S + jc) * scl;
                bad |= !isfinite(v);
                orow[jc] = v;
              }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)F8_N) : "memory");
  }
}

__global__ void fp8_reduce_kernel(const float* part, int P, int64_t pstride, int l, int64_t n, float* X,
                                  int64_t ldx, float scale, int32_t* dev_status) {
  bool bad = false;
  for (int r = blockIdx.y; r < l; r += gridDim.y)
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
      const int64_t e = (int64_t)r * n + c;
      float a = 0.f;
      for (int q = 0; q < P; ++q) a += part[q * pstride + e];
      const float v = a * scale;
      bad |= !isfinite(v);
      X[(int64_t)r * ldx + c] = v;
    }
  if (bad) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
}

struct F8Plan {
  int lblocks, jtiles, P;
  int64_t nkb, ld8, mg, lp;
};

F8Plan plan_f8(int64_t m, int64_t n, int l) {
  F8Plan pl{};
  pl.lblocks = (l + 127) / 128;
  pl.jtiles = (int)((n + F8_N - 1) / F8_N);
  pl.nkb = (m + F8_BLOCK - 1) / F8_BLOCK;
  pl.ld8 = (m + 15) / 16 * 16;
  pl.mg = pl.nkb * F8_BLOCK;
  pl.lp = (int64_t)pl.lblocks * 128;
  const int sms = device_sm_count();
  int P = std::max(1, sms / std::max(1, pl.lblocks * pl.jtiles));
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, pl.nkb / 4));
  pl.P = std::min(P, 16);
  return pl;
}

}  // namespace

size_t sketch_fp8_workspace(int64_t m, int64_t n, int32_t l) {
  const F8Plan pl = plan_f8(m, n, l);
  return align_up((size_t)pl.ld8 * n) + align_up(sizeof(float) * (size_t)n) +
         align_up((size_t)pl.lp * pl.mg) + (pl.P > 1 ? align_up(sizeof(float) * (size_t)pl.P * l * n) : 0);
}

cudaError_t launch_sketch_fp8(int64_t row0, int64_t m, int64_t n, const float* A, int64_t lda, int32_t l,
                              uint64_t seed, float* X, int64_t ldx, void* ws, int32_t* dev_status, cudaStream_t st) {
  if (row0 != 0) return cudaErrorNotSupported;    // Gamma columns from 0: no row-block offset here
  if (m < 1 || n < 1 || m > (int64_t)INT32_MAX || n > (int64_t)INT32_MAX) return cudaErrorNotSupported;
  if ((lda % 4) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const F8Plan pl = plan_f8(m, n, l);
  unsigned char* base = static_cast<unsigned char*>(ws);
  uint8_t* A8 = base;
  base += align_up((size_t)pl.ld8 * n);
  float* S = reinterpret_cast<float*>(base);
  base += align_up(sizeof(float) * (size_t)n);
  uint8_t* G8 = base;
  base += align_up((size_t)pl.lp * pl.mg);
  float* part = reinterpret_cast<float*>(base);
  CUtensorMap tA, tG;
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)pl.ld8};
    const cuuint32_t box[2] = {F8_BLOCK, 256};           // two boxes per 512-column tile
    const cuuint32_t es[2] = {1, 1};
    if (enc(&tA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, A8, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)pl.mg, (cuuint64_t)pl.lp};
    const cuuint64_t gstride[1] = {(cuuint64_t)pl.mg};
    const cuuint32_t box[2] = {F8_BLOCK, 128};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&tG, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, G8, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  const int sms = device_sm_count();
  {
    KernelTimer kt("fp8_quantize", st);
    // two CTAs per SM: a few hundred columns in flight, so that each column's second read hits L2
    fp8_quantize_kernel<<<(unsigned)std::min<int64_t>(n, 2 * sms), 512, 0, st>>>(m, n, A, lda, A8, pl.ld8, S,
                                                                                 dev_status);
  }
  fp8_gamma_kernel<<<(unsigned)std::min<int64_t>((pl.lp * pl.mg / 4 + 255) / 256, 4096), 256, 0, st>>>(
      l, (int)pl.lp, m, pl.mg, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), G8);
  note_launches(2);
  F8Params p{};
  p.m = m; p.n = n; p.l = l; p.P = pl.P; p.nkb = pl.nkb;
  p.S = S;
  p.direct = pl.P == 1;
  p.scale = (float)(1.0 / std::sqrt((double)l));
  p.out = p.direct ? X : part;
  p.ldo = p.direct ? ldx : n;
  p.part_stride = (int64_t)l * n;
  p.dev_status = dev_status;
  cudaError_t e = cudaFuncSetAttribute(sketch_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F8_SMEM);
  if (e != cudaSuccess) return e;
  {
    KernelTimer kt("sketch_fp8", st);
    sketch_fp8_kernel<<<dim3(pl.lblocks, pl.jtiles, pl.P), F8_THREADS, F8_SMEM, st>>>(tA, tG, p);
  }
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || p.direct) return e;
  fp8_reduce_kernel<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(l, 128)), 256, 0, st>>>(
      part, pl.P, p.part_stride, l, n, X, ldx, p.scale, dev_status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
