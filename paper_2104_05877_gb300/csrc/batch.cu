// Batched skeletonization of many independent blocks (hierarchical-matrix compression): per
// block A_b (m_b x n_b, FP32, column-major) the Gaussian sketch X_b = Gamma A_b (Algorithm 2),
// column LUPP on X_b (Sec. 2.5.2, Algorithm 2) stopped at the tolerance-driven rank r, and
// the column ID coefficients formed from the sketch alone (C^+ A ~ X_1^+ X, Sec. 4, ID
// without a second pass over A), the pseudo-inverse over all l rows of the sketch:
//   Z_b = X_b(:, J)^+ X_b = argmin_Z ||X_b(:, J) Z - X_b||_F.
// A is read once.
//
// Kernels, all launched by skel_batch_run on the caller's stream:
//   batch_gamma_kernel   the standard normals G (l x m_max, one Gamma for every block: the
//                        blocks are independent problems and each sees a Gaussian sketch),
//                        split into TF32 halves G = Ghi + Glo; 2 l m_max floats that stay in L2.
//   batch_sketch_kernel  one CTA per 128-column tile of a block: tcgen05 kind::tf32 with
//                        M = 128 columns of A_b (A operand, K-major as A is stored) and
//                        N = l_pad rows of Gamma (B operand); both operands split into TF32
//                        halves (A in shared memory as it arrives) and X = Ahi Ghi +
//                        (Ahi Glo + Alo Ghi) in two TMEM accumulators, so X carries FP32
//                        accuracy (the interpolation Z inherits the sketch's precision).
//   batch_lupp_kernel    one cluster of CL in {1, 2, 4} CTAs per block, each CTA holding the
//                        block's X for n_b/CL columns in shared memory: per step every CTA
//                        sends its best candidate (with the candidate's full column) and the
//                        sum of squares of its rows below the step to every CTA through
//                        distributed shared memory, one cluster barrier, then every CTA
//                        takes the same decision (stop at the tolerance rank, or the pivot)
//                        and updates its columns.  Writes J and the rank.
//   batch_lsq_kernel     one CTA per block: Householder QR of X_b(:, J) (l x r) in shared
//                        memory, Q^T applied to X_b in chunks of columns, back substitution
//                        with R; Z_b(:, J) = I exactly.
// The tolerance rule (the paper fixes k): the rank is the smallest t <= k_max with
//   ||S_t||_F^2 l/(l - t) <= tol^2 ||X||_F^2,
// S_t the Schur complement (rows t..l-1) after t steps, an unbiased estimate of
// ||A (I - P_t)||_F^2 >= ||A - C C^+ A||_F^2 (proof of Theorem 1), or k_max.
#include <cooperative_groups.h>
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace cg = cooperative_groups;

struct skel_batch_plan;

namespace skel {

namespace {

using namespace tc;

struct BatchBlock {
  const float* A;   // A_b (column-major, lda); for a point plan the records of x_1 .. x_m
  int64_t lda;
  int32_t m, n;
  int64_t xoff;     // X_b at X + xoff (l x n_b row-major)
  int64_t zoff;     // Z_b at Z + zoff (k_max x n_b row-major)
  const float* Y;   // point plans: the records of y_1 .. y_n
};

// A point record (point plans): 8 floats, {p_0, p_1, p_2, 0, c_hi, c_lo, 0, 0} with the
// coordinates padded by zeros to three and c = -||p||^2 / h^2 as an unevaluated sum of two
// floats (formed in FP64).
constexpr int kRec = 8;
struct SketchItem {
  int32_t b, tile;
};

// ---------------------------------------------------------------------------------------
// Gamma halves
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void batch_gamma_kernel(int l, int lp, int64_t mg, uint32_t k0, uint32_t k1, float* Ghi, float* Glo) {
  const int64_t m4 = mg / 4;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)lp * m4;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m4);
    const int64_t j4 = e % m4;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < l) g = gaussian4_f32(k0, k1, (uint32_t)i, (uint32_t)j4);
    const float v[4] = {g.x, g.y, g.z, g.w};
    float4 h, lo;
    float* hp = &h.x;
    float* lp_ = &lo.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hp[q] = tf32_rna(v[q]);
      lp_[q] = tf32_rna(v[q] - hp[q]);
    }
    reinterpret_cast<float4*>(Ghi + (int64_t)i * mg)[j4] = h;
    reinterpret_cast<float4*>(Glo + (int64_t)i * mg)[j4] = lo;
  }
}

// ---------------------------------------------------------------------------------------
// Sketch: X_b(:, tile) = Gamma A_b(:, tile), 3xTF32
// ---------------------------------------------------------------------------------------
constexpr int BS_THREADS = 256;       // warp 0 TMA, 1 MMA, 2 TMEM, 4..7 converters + epilogue
constexpr int BS_THREADS_P = 384;     // point plans: warps 4..11 generate A's tiles, 4..7 epilogue
constexpr int BS_CONV_WARP0 = 4;
constexpr int BS_BK = 32;
constexpr uint32_t BS_ATILE = 128 * 128;          // 128 columns x 32 rows of A, FP32
constexpr uint32_t BS_CORR_COL = 256;             // TMEM column of the correction accumulator
constexpr uint32_t BS_XREC = 32 * 32;              // point plans: the 32 x records of a step
constexpr uint64_t BS_WAIT_NS = 2000000000ull;

struct BatchSketchParams {
  const BatchBlock* blocks;
  const CUtensorMap* tmaps;   // one per block, in global memory (64-byte aligned); stored blocks
  const SketchItem* items;
  float* X;
  int l, lp, stages;
  float scale;
  float w_hi, w_lo;           // point plans: 2 / h^2 as an unevaluated sum of two floats
  int32_t* dev_status;
};

// Two-sum (Knuth): s + e = a + b exactly, s = fl(a + b).  Explicit round-to-nearest
// operations, so that no multiply-add contraction alters the error terms.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Gaussian-kernel entry exp(-||x - y||^2 / h^2) from two point records, through
//   -||x - y||^2 / h^2 = c_x + c_y + (2 / h^2) x.y,   c_p = -||p||^2 / h^2,
// evaluated as an unevaluated sum of two floats (products split exactly with FMA, sums by
// two-sum), so the exponent carries ~44 bits: a plain FP32 evaluation would put an absolute
// error of ~1e-5 into exponents near -100 and a relative error of that size into the entry.
// The entry is expf(a_hi) (1 + a_lo).
__device__ __forceinline__ float kernel_entry(const float4 x, const float2 cx, const float4 y, const float2 cy,
                                              float w_hi, float w_lo) {
  const float p0 = __fmul_rn(x.x, y.x), p1 = __fmul_rn(x.y, y.y), p2 = __fmul_rn(x.z, y.z);
  const float e0 = fmaf(x.x, y.x, -p0), e1 = fmaf(x.y, y.y, -p1), e2 = fmaf(x.z, y.z, -p2);
  float s1, t1, dh, t2;
  two_sum(p0, p1, s1, t1);
  two_sum(s1, p2, dh, t2);
  const float dl = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, t1)), t2);   // x.y = dh + dl
  const float ph = __fmul_rn(dh, w_hi);
  const float pl = fmaf(dh, w_lo, fmaf(dl, w_hi, fmaf(dh, w_hi, -ph)));               // w x.y = ph + pl
  float u, ue, ah, ae;
  two_sum(cx.x, cy.x, u, ue);
  two_sum(u, ph, ah, ae);
  const float al = __fadd_rn(__fadd_rn(__fadd_rn(ue, ae), __fadd_rn(cx.y, cy.y)), pl);
  const float ex = expf(ah);
  return fmaf(ex, al, ex);
}

// Point records of every block (one grid row per block), formed at the start of each run from
// the caller's points (m_b x dim and n_b x dim, row-major FP32, dim <= 3).
struct PointSrc {
  const float* x;
  const float* y;
  int32_t m, n;
  float* xrec;
  float* yrec;
};

__global__ void batch_points_prep_kernel(const PointSrc* src, int dim, double inv_h2) {
  const PointSrc ps = src[blockIdx.y];
  const int tot = ps.m + ps.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const bool isx = e < ps.m;
    const int i = isx ? e : e - ps.m;
    const float* q = (isx ? ps.x : ps.y) + (int64_t)i * dim;
    float c3[3] = {0.f, 0.f, 0.f};
    double n2 = 0.0;
    for (int d = 0; d < dim; ++d) {
      c3[d] = q[d];
      n2 += (double)c3[d] * (double)c3[d];
    }
    const double c = -n2 * inv_h2;
    const float ch = (float)c;
    const float cl = (float)(c - (double)ch);
    float4* r = reinterpret_cast<float4*>((isx ? ps.xrec : ps.yrec) + (int64_t)i * kRec);
    r[0] = make_float4(c3[0], c3[1], c3[2], 0.f);
    r[1] = make_float4(ch, cl, 0.f, 0.f);
  }
}

// PTS: the block is given by point records and the generator warps form A's tiles in shared
// memory (in the 128-byte swizzled K-major layout the TMA would have written), so A is never
// read from (or stored in) device memory.
template <bool PTS>
__global__ void __launch_bounds__(PTS ? BS_THREADS_P : BS_THREADS, 1)
batch_sketch_kernel(const __grid_constant__ CUtensorMap tmGhi, const __grid_constant__ CUtensorMap tmGlo,
                    const BatchSketchParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int AS = p.stages;
  const uint32_t g_bytes = (uint32_t)p.lp * 128;
  // [Ahi][Alo][Ghi][Glo] (+ [x records of the step] for point plans; 1 KB keeps 1024-byte alignment)
  const uint32_t stage_bytes = 2 * BS_ATILE + 2 * g_bytes + (PTS ? BS_XREC : 0u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + AS * stage_bytes);   // full, conv, empty [AS]; done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * AS + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const SketchItem item = p.items[blockIdx.x];
  const BatchBlock blk = p.blocks[item.b];
  const CUtensorMap* tmA = PTS ? nullptr : p.tmaps + item.b;
  const int nk = (blk.m + BS_BK - 1) / BS_BK;
  constexpr int kConvWarps = PTS ? (BS_THREADS_P / 32 - BS_CONV_WARP0) : 4;
  auto a_buf = [&](int s) { return smem + s * stage_bytes; };
  auto alo_buf = [&](int s) { return smem + s * stage_bytes + BS_ATILE; };
  auto ghi_buf = [&](int s) { return smem + s * stage_bytes + 2 * BS_ATILE; };
  auto glo_buf = [&](int s) { return smem + s * stage_bytes + 2 * BS_ATILE + g_bytes; };
  auto xr_buf = [&](int s) { return smem + s * stage_bytes + 2 * BS_ATILE + 2 * g_bytes; };
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto conv = [&](int s) { return smem_u32(&bars[AS + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * AS + s]); };
  const uint32_t done = smem_u32(&bars[3 * AS]);

  if (tid == 0) {
    for (int s = 0; s < AS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), kConvWarps);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(512u) : "memory");
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
        const int s = it % AS;
        const uint32_t ph = (uint32_t)(it / AS) & 1u;
        if (aborted()) break;
        if (it >= AS && !mbar_wait(empty(s), ph ^ 1u, BS_WAIT_NS)) { fail(); break; }
        mbar_expect_tx(full(s), (PTS ? BS_XREC : BS_ATILE) + 2 * g_bytes);
        const int x = it * BS_BK;
        if constexpr (PTS)
          bulk_load_g2s(smem_u32(xr_buf(s)), blk.A + (int64_t)x * kRec, BS_XREC, full(s));   // the step's x records
        else
          tma_load_2d(smem_u32(a_buf(s)), tmA, x, item.tile * 128, full(s));
        tma_load_2d(smem_u32(ghi_buf(s)), &tmGhi, x, 0, full(s));
        tma_load_2d(smem_u32(glo_buf(s)), &tmGlo, x, 0, full(s));
        ++issued;
      }
      for (int it = std::max(0, issued - AS); it < issued; ++it)
        if (!mbar_wait(full(it % AS), (uint32_t)(it / AS) & 1u, BS_WAIT_NS)) fail();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, p.lp);
      for (int it = 0; it < nk; ++it) {
        const int s = it % AS;
        const uint32_t ph = (uint32_t)(it / AS) & 1u;
        if (aborted()) break;
        if (PTS && !mbar_wait(full(s), ph, BS_WAIT_NS)) { fail(); break; }   // Gamma's tiles
        if (!mbar_wait(conv(s), ph, BS_WAIT_NS)) { fail(); break; }
        tc_fence_after();
        const uint32_t ahi = smem_u32(a_buf(s)), alo = smem_u32(alo_buf(s));
        const uint32_t ghi = smem_u32(ghi_buf(s)), glo = smem_u32(glo_buf(s));
#pragma unroll
        for (int kk = 0; kk < BS_BK / 8; ++kk) {
          const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(tmem, sw128_desc(ahi + kk * 32), sw128_desc(ghi + kk * 32), idesc, acc);
          mma_tf32(tmem + BS_CORR_COL, sw128_desc(ahi + kk * 32), sw128_desc(glo + kk * 32), idesc, acc);
          mma_tf32(tmem + BS_CORR_COL, sw128_desc(alo + kk * 32), sw128_desc(ghi + kk * 32), idesc, 1u);
        }
        mma_commit(empty(s));
      }
      mma_commit(done);
    }
  } else if (warp >= BS_CONV_WARP0) {
    if constexpr (PTS) {
      // generators: thread gt forms column jl of the tile (y_j) for the k-chunks 4hh .. 4hh+3
      // of every 32-row step: A(i, j) for i = 32 it + 4c + u, split into TF32 halves and
      // stored as 16-byte chunk c of row jl (swizzled: chunk c ^ (jl mod 8)).  The x records
      // of a step are the same for the 32 lanes of a warp (broadcast loads).
      const int gt = tid - BS_CONV_WARP0 * 32;        // 0..255
      const int jl = gt & 127, hh = gt >> 7;
      const int64_t j = (int64_t)item.tile * 128 + jl;
      const bool colv = j < blk.n;
      float4 yc = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 cy = make_float2(0.f, 0.f);
      if (colv) {
        const float4* yr = reinterpret_cast<const float4*>(blk.Y + j * kRec);
        yc = __ldg(yr);
        const float4 t = __ldg(yr + 1);
        cy = make_float2(t.x, t.y);
      }
      for (int it = 0; it < nk; ++it) {
        const int s = it % AS;
        const uint32_t ph = (uint32_t)(it / AS) & 1u;
        if (aborted()) break;
        if (it >= AS && !mbar_wait(empty(s), ph ^ 1u, BS_WAIT_NS)) { fail(); break; }
        if (!mbar_wait(full(s), ph, BS_WAIT_NS)) { fail(); break; }     // the step's x records
        float4* ahi = reinterpret_cast<float4*>(a_buf(s));
        float4* alo = reinterpret_cast<float4*>(alo_buf(s));
        const float4* xs = reinterpret_cast<const float4*>(xr_buf(s));
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = 4 * hh + cc;
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = it * BS_BK + 4 * c + u;
            v[u] = 0.f;
            if (colv && i < blk.m) {
              const float4 xc = xs[2 * (4 * c + u)];
              const float4 t = xs[2 * (4 * c + u) + 1];
              v[u] = kernel_entry(xc, make_float2(t.x, t.y), yc, cy, p.w_hi, p.w_lo);
            }
          }
          float4 h, w;
          h.x = tf32_rna(v[0]); w.x = tf32_rna(v[0] - h.x);
          h.y = tf32_rna(v[1]); w.y = tf32_rna(v[1] - h.y);
          h.z = tf32_rna(v[2]); w.z = tf32_rna(v[2] - h.z);
          h.w = tf32_rna(v[3]); w.w = tf32_rna(v[3] - h.w);
          const int pos = jl * 8 + (c ^ (jl & 7));
          ahi[pos] = h;
          alo[pos] = w;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(conv(s));
      }
    }
    // converters: A tile -> Ahi in place, Alo beside it (same positions: swizzle-agnostic)
    const int ct = tid - BS_CONV_WARP0 * 32;          // 0..127
    for (int it = 0; !PTS && it < nk; ++it) {
      const int s = it % AS;
      const uint32_t ph = (uint32_t)(it / AS) & 1u;
      if (aborted()) break;
      if (!mbar_wait(full(s), ph, BS_WAIT_NS)) { fail(); break; }
      float4* a = reinterpret_cast<float4*>(a_buf(s));
      float4* lo = reinterpret_cast<float4*>(alo_buf(s));
#pragma unroll
      for (int q = 0; q < (int)(BS_ATILE / 16) / 128; ++q) {
        const int e = ct + 128 * q;
        const float4 v = a[e];
        float4 h, w;
        h.x = tf32_rna(v.x); w.x = tf32_rna(v.x - h.x);
        h.y = tf32_rna(v.y); w.y = tf32_rna(v.y - h.y);
        h.z = tf32_rna(v.z); w.z = tf32_rna(v.z - h.z);
        h.w = tf32_rna(v.w); w.w = tf32_rna(v.w - h.w);
        a[e] = h;
        lo[e] = w;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(conv(s));
    }
    // epilogue (warps 4..7): lane = column of the tile, TMEM columns = rows of X
    const bool ok = warp < BS_CONV_WARP0 + 4 && mbar_wait(done, 0, BS_WAIT_NS);
    if (!ok && warp < BS_CONV_WARP0 + 4) fail();
    tc_fence_after();
    if (ok && !aborted()) {
      const int qd = warp & 3;
      const int64_t j = (int64_t)item.tile * 128 + qd * 32 + lane;
      float* xb = p.X + blk.xoff;
      bool bad = false;
      for (int c0 = 0; c0 < p.lp; c0 += 32) {
        uint32_t rm[32], rc[32];
        TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, rm);
        TMEM_LD32(tmem + ((uint32_t)(qd * 32) << 16) + BS_CORR_COL + (uint32_t)c0, rc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j < blk.n) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int i = c0 + q;
            if (i < p.l) {
              const float v = (__uint_as_float(rm[q]) + __uint_as_float(rc[q])) * p.scale;
              bad |= !isfinite(v);
              xb[(int64_t)i * blk.n + j] = v;
            }
          }
        }
      }
      if (bad) record_error(p.dev_status, SKEL_ERR_NONFINITE, -1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// Tolerance-rank LUPP on X_b and Z_b = R_1^{-1} R
// ---------------------------------------------------------------------------------------
constexpr int BL_THREADS = 512;
constexpr int BL_MAXCL = 4;
constexpr int BL_MAXL = 256;
constexpr int BL_MAXK = 128;

struct __align__(16) BlSlot {
  float col[BL_MAXL];     // the candidate's column, rows 0 .. l-1
  float nu;               // sender's sum of squares of the rows below the step
  float key;              // |S(t, j)|, -1 when the sender has no candidate
  int idx;                // global column index, INT_MAX when none
};

struct BatchLuppParams {
  const BatchBlock* blocks;
  const int32_t* order;   // block handled by each cluster
  const float* X;
  int l, kmax;
  float tol2;
  int32_t* Js;            // nblocks x kmax
  int32_t* ranks;
  int32_t* dev_status;
};

__device__ __forceinline__ int bl_ldp(int ncl) { return (ncl & 1) ? ncl : ncl + 1; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// The stopping rule is tested without a division: nu_t l <= tol^2 ||X||^2 (l - t).  Sums of
// squares have no cancellation, so FP32 carries them.
__global__ void __launch_bounds__(BL_THREADS, 1) batch_lupp_kernel(const BatchLuppParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BlSlot slot[2][BL_MAXCL];
  __shared__ float s_amax[BL_MAXCL];
  __shared__ int s_J[BL_MAXK];
  __shared__ float wkey[BL_THREADS / 32];
  __shared__ int widx[BL_THREADS / 32];
  __shared__ float wnu[BL_THREADS / 32];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), crank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = p.order[blockIdx.x / CL];
  const BatchBlock blk = p.blocks[b];
  const int n = blk.n, l = p.l, kmax = p.kmax;
  const int ncl = (n + CL - 1) / CL;
  const int c0 = crank * ncl;
  const int nl = max(0, min(ncl, n - c0));
  const int ldp = bl_ldp(ncl);
  float* S = reinterpret_cast<float*>(smem);                 // [l][ldp]
  unsigned char* sel = reinterpret_cast<unsigned char*>(S + (size_t)l * ldp);        // [ncl]
  const float* xb = p.X + blk.xoff;


  // The block's X is scaled by the power of two that brings its largest magnitude into
  // [1, 2): exact in FP32, so pivots and ranks do not change, but the squares of Schur
  // complement entries near the tolerance stay far above FP32's underflow threshold (kernel
  // blocks between distant clusters have entries near 1e-13, whose tolerance-level residues
  // would square to ~1e-38).  The scale is agreed across the cluster.
  float am = 0.f;
  for (int e0 = tid; e0 < l * nl; e0 += 8 * BL_THREADS) {   // eight loads in flight per thread
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * BL_THREADS;
      v[u] = e < l * nl ? xb[(int64_t)(e / nl) * n + c0 + e % nl] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * BL_THREADS;
      if (e < l * nl) {
        S[(e / nl) * ldp + e % nl] = v[u];
        am = fmaxf(am, fabsf(v[u]));    // NaN is ignored here and flagged by the pivot search
      }
    }
  }
  for (int jl = tid; jl < nl; jl += BL_THREADS) sel[jl] = 0;
  am = warp_max(am);
  if (lane == 0) wnu[warp] = am;
  cluster.sync();                        // every CTA of the cluster is running before DSMEM writes
  if (tid == 0) {
    float a = 0.f;
    for (int w = 0; w < BL_THREADS / 32; ++w) a = fmaxf(a, wnu[w]);
    for (int d = 0; d < CL; ++d) *cluster.map_shared_rank(&s_amax[crank], d) = a;
  }
  cluster.sync();
  float amax = 0.f;
  for (int d = 0; d < CL; ++d) amax = fmaxf(amax, s_amax[d]);
  const float sc = amax > 0.f && amax < INFINITY ? ldexpf(1.f, -ilogbf(amax)) : 1.f;
  // Sums of squares: FP32 per thread over its entries, then warp sums and the warps' sum in a
  // fixed order.  A thread's partial for step t is over the entries it updated at step t-1
  // (all its entries at t = 0), so ||S_t||^2 rides with step t's candidate reduction.
  float nuloc = 0.f;
  for (int e = tid; e < l * nl; e += BL_THREADS) {
    const int r = e / nl, jl = e % nl;
    const float v = S[r * ldp + jl] * sc;
    S[r * ldp + jl] = v;
    nuloc = fmaf(v, v, nuloc);
  }
  __syncthreads();

  // Per step one CTA barrier (the candidates and sums of squares of the warps) and one
  // cluster barrier (the CTAs' candidates); every thread then takes the same decision from
  // the same slots in the same order.
  int rank = 0, code = 0;
  float normX2 = 0.f;
  for (int t = 0;; ++t) {
    // this CTA's candidate on row t: largest magnitude, ties to the lower column index
    float key = -1.f;
    int idx = INT_MAX;
    for (int jl = tid; jl < nl; jl += BL_THREADS) {
      if (sel[jl]) continue;
      const float a = fabsf(S[t * ldp + jl]);
      const float k = a == a ? a : INFINITY;     // NaN is flagged as non-finite below
      if (k > key) { key = k; idx = c0 + jl; }
    }
    const int par = t & 1;
    float nu_cta;
    {
      const unsigned kb = key >= 0.f ? __float_as_uint(key) : 0u;
      const unsigned m = __reduce_max_sync(0xffffffffu, kb);
      const unsigned im = __reduce_min_sync(0xffffffffu, kb == m && key >= 0.f ? (unsigned)idx : 0x7fffffffu);
      const float nw_ = warp_sum(nuloc);
      if (lane == 0) {
        wkey[warp] = im == 0x7fffffffu ? -1.f : __uint_as_float(m);
        widx[warp] = (int)im;
        wnu[warp] = nw_;
      }
      __syncthreads();
      float k2 = lane < BL_THREADS / 32 ? wkey[lane] : -1.f;
      int i2 = lane < BL_THREADS / 32 ? widx[lane] : 0x7fffffff;
      const unsigned kb2 = k2 >= 0.f ? __float_as_uint(k2) : 0u;
      const unsigned m2 = __reduce_max_sync(0xffffffffu, kb2);
      const unsigned im2 = __reduce_min_sync(0xffffffffu, kb2 == m2 && k2 >= 0.f ? (unsigned)i2 : 0x7fffffffu);
      key = im2 == 0x7fffffffu ? -1.f : __uint_as_float(m2);
      idx = im2 == 0x7fffffffu ? INT_MAX : (int)im2;
      float a = 0.f;
      for (int w = 0; w < BL_THREADS / 32; ++w) a += wnu[w];
      nu_cta = a;
    }
    // send it (with its whole column and this CTA's sum of squares) to every CTA
    const bool have = idx != INT_MAX;
    for (int d = 0; d < CL; ++d) {
      BlSlot* dst = cluster.map_shared_rank(&slot[par][crank], d);
      for (int r = tid; r < l; r += BL_THREADS) dst->col[r] = have ? S[r * ldp + (idx - c0)] : 0.f;
      if (tid == 0) {
        dst->nu = nu_cta;
        dst->key = key;
        dst->idx = idx;
      }
    }
    cluster.sync();
    // the same decision in every thread of every CTA (the same inputs, summed in CTA order)
    float nut = 0.f;
    for (int d = 0; d < CL; ++d) nut += slot[par][d].nu;
    if (t == 0) normX2 = nut;
    float bk = -1.f;
    int bi = INT_MAX, o = 0;
    for (int d = 0; d < CL; ++d) {
      const float k = slot[par][d].key;
      const int i = slot[par][d].idx;
      if (i != INT_MAX && (k > bk || (k == bk && i < bi))) { bk = k; bi = i; o = d; }
    }
    const bool stop = nut * (float)l <= p.tol2 * normX2 * (float)(l - t) || t >= kmax || bi == INT_MAX ||
                      !(bk > 0.f) || !isfinite(bk);
    if (stop) {
      rank = t;
      code = bi != INT_MAX && !isfinite(bk) ? SKEL_ERR_NONFINITE : 0;
      break;
    }
    const float* pc = slot[par][o].col;
    const float piv = pc[t];
    if (tid == 0) s_J[t] = bi;
    // The pivot column leaves the candidates: the thread that scans it marks it (its entries
    // below row t would become exact zeros and are not read again, so whether an updating
    // thread still sees it unmarked changes nothing).
    if (o == crank && (bi - c0) % BL_THREADS == tid) sel[bi - c0] = 1;
    // rows t+1 .. l-1 of the local columns: S(r, j) -= S(r, j_t) S(t, j) / pivot
    nuloc = 0.f;
    if (nl > 0) {
      const int nph = max(1, BL_THREADS / nl);           // threads per column (rows split)
      for (int e = tid; e < nph * nl; e += BL_THREADS) {
        const int jl = e % nl, ph = e / nl;
        if (sel[jl]) continue;
        const float rv = S[t * ldp + jl] / piv;
        float* col = S + jl;
        int r = t + 1 + ph;
        for (; r + 3 * nph < l; r += 4 * nph) {         // four rows' loads in flight
          float x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = col[(r + u * nph) * ldp];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            x[u] = __fsub_rn(x[u], __fmul_rn(pc[r + u * nph], rv));
            col[(r + u * nph) * ldp] = x[u];
            nuloc = fmaf(x[u], x[u], nuloc);
          }
        }
        for (; r < l; r += nph) {
          const float x = __fsub_rn(col[r * ldp], __fmul_rn(pc[r], rv));
          col[r * ldp] = x;
          nuloc = fmaf(x, x, nuloc);
        }
      }
    }
  }
  if (crank == 0) {
    for (int q = tid; q < kmax; q += BL_THREADS) p.Js[(int64_t)b * kmax + q] = q < rank ? s_J[q] : -1;
    if (tid == 0) {
      p.ranks[b] = rank;
      if (code) record_error(p.dev_status, code, b);
    }
  }
}

size_t lupp_smem(int l, int kmax, int ncl) {
  (void)kmax;
  const int ldp = (ncl & 1) ? ncl : ncl + 1;
  return sizeof(float) * (size_t)l * ldp + (size_t)ncl;
}

// ---------------------------------------------------------------------------------------
// Z_b = X_b(:, J)^+ X_b (l x n_b sketch, r = rank_b pivots): FP32 Householder QR of the l x r
// X_b(:, J) in shared memory (column-major, odd leading dimension), then for each chunk of
// LS_NC columns of X_b: Q^T applied four reflectors at a time in compact WY form,
// (H_t .. H_t+3)^T x = x - V_4 T_4^T V_4^T x with T_4 (4 x 4) formed once per group
// (LS_TPC threads per column, rows split by residue: one pass for the four dot products, one
// for the update), then the back substitution with R, column-oriented over the same eight
// lanes.  Z(:, J) = I is written exactly.
constexpr int LS_THREADS = 256;
constexpr int LS_NC = 32;                          // columns per chunk
constexpr int LS_TPC = LS_THREADS / LS_NC;         // threads per column (a power of two <= 32)

struct BatchLsqParams {
  const BatchBlock* blocks;
  const float* X;
  int l, kmax;
  const int32_t* Js;
  const int32_t* ranks;
  double* Z;
  int32_t* dev_status;
};

__host__ __device__ __forceinline__ int ls_ld(int l) { return (l & 1) ? l : l + 1; }

size_t lsq_smem(int l, int kmax) { return sizeof(float) * (size_t)ls_ld(l) * (kmax + LS_NC); }

__global__ void __launch_bounds__(LS_THREADS) batch_lsq_kernel(const BatchLsqParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float tau[BL_MAXK];
  __shared__ float rdiag[BL_MAXK];                      // R(t, t); V(t, t) holds the reflector's 1
  __shared__ float T4[BL_MAXK / 4][16];                 // per group of four: T_4 (row-major)
  __shared__ float red[LS_THREADS / 32];
  __shared__ float s_nrm2;
  const int b = blockIdx.x;
  const BatchBlock blk = p.blocks[b];
  const int r = p.ranks[b];
  if (r <= 0) return;
  const int n = blk.n, l = p.l, ldv = ls_ld(l);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t* J = p.Js + (int64_t)b * p.kmax;
  const float* xb = p.X + blk.xoff;
  double* zb = p.Z + blk.zoff;
  float* V = reinterpret_cast<float*>(smem);             // [kmax][ldv]: column t of X(:, J), then v_t / R
  float* Cc = V + (size_t)p.kmax * ldv;                  // [LS_NC][ldv]: a chunk of X's columns

  float amax = 0.f;
  for (int e0 = tid; e0 < l * r; e0 += 8 * LS_THREADS) {    // eight loads in flight per thread
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * LS_THREADS;
      x[u] = 0.f;
      if (e < l * r) {
        const int j = J[e / l];
        x[u] = j >= 0 && j < n ? xb[(int64_t)(e % l) * n + j] : __int_as_float(0x7fc00000);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * LS_THREADS;
      if (e < l * r) {
        V[(e / l) * ldv + e % l] = x[u];
        amax = fmaxf(amax, fabsf(x[u]));
      }
    }
  }
  // Z = X(:, J)^+ X does not change when X is scaled, so X is scaled by the power of two that
  // brings max |X(:, J)| into [0.5, 1) (exact): blocks far apart in a kernel matrix have
  // entries near 1e-28, whose squares in the reflectors' norms would underflow FP32.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (lane == 0) red[warp] = amax;
  __syncthreads();
  if (tid == 0) {
    float a = 0.f;
    for (int w = 0; w < LS_THREADS / 32; ++w) a = fmaxf(a, red[w]);
    s_nrm2 = a;
  }
  __syncthreads();
  int sh = 0;
  if (s_nrm2 > 0.f && isfinite(s_nrm2)) {
    frexpf(s_nrm2, &sh);
    sh = -sh;
  }
  for (int e = tid; e < l * r; e += LS_THREADS) {
    const int t = e / l, i = e % l;
    V[t * ldv + i] = ldexpf(V[t * ldv + i], sh);
  }
  __syncthreads();
  // Householder QR: H_t = I - tau_t v v^T with v(t) = 1, R(t, t) = beta = -sign(alpha) ||x||
  for (int t = 0; t < r; ++t) {
    float* v = V + t * ldv;
    float part = 0.f;
    for (int i = t + tid; i < l; i += LS_THREADS) part = fmaf(v[i], v[i], part);
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      float a = 0.f;
      for (int w = 0; w < LS_THREADS / 32; ++w) a += red[w];
      s_nrm2 = a;
    }
    __syncthreads();
    const float nrm2 = s_nrm2, alpha = v[t];
    const float beta = alpha >= 0.f ? -sqrtf(nrm2) : sqrtf(nrm2);
    const bool refl = nrm2 > 0.f;
    __syncthreads();                                     // every thread has read v[t]
    if (refl)
      for (int i = t + 1 + tid; i < l; i += LS_THREADS) v[i] = v[i] / (alpha - beta);
    if (tid == 0) {
      tau[t] = refl ? (beta - alpha) / beta : 0.f;
      v[t] = beta;
      rdiag[t] = beta;
    }
    __syncthreads();
    const float tt = tau[t];
    for (int c = t + 1 + warp; c < r; c += LS_THREADS / 32) {   // one warp per later column
      float* x = V + c * ldv;
      float d = lane == 0 ? x[t] : 0.f;
      for (int i = t + 1 + lane; i < l; i += 32) d = fmaf(v[i], x[i], d);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      d *= tt;
      if (lane == 0) x[t] -= d;
      for (int i = t + 1 + lane; i < l; i += 32) x[i] = fmaf(-d, v[i], x[i]);
    }
    __syncthreads();
  }
  // the reflectors' unit diagonal in V (R's diagonal is in rdiag), then T_4 per group of four:
  // T(j, j) = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j), G(i, j) = v_i^T v_j
  for (int t = tid; t < r; t += LS_THREADS) V[t * ldv + t] = 1.f;
  __syncthreads();
  const int ng = (r + 3) / 4;
  for (int g = warp; g < ng; g += LS_THREADS / 32) {
    const int t0 = 4 * g, nw4 = min(4, r - t0);
    float G[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float d = 0.f;
        if (a < c && c < nw4) {        // v_a(i) = 0 for i < t0 + a; v_c(i) = 0 for i < t0 + c
          const float* va = V + (t0 + a) * ldv;
          const float* vc = V + (t0 + c) * ldv;
          for (int i = t0 + c + lane; i < l; i += 32) d = fmaf(va[i], vc[i], d);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        G[a][c] = d;
      }
    if (lane == 0) {
      float Tm[4][4] = {};
      for (int j = 0; j < nw4; ++j) {
        const float tj = tau[t0 + j];
        Tm[j][j] = tj;
        for (int i = 0; i < j; ++i) {
          float a = 0.f;
          for (int k = i; k < j; ++k) a = fmaf(Tm[i][k], G[k][j], a);
          Tm[i][j] = -tj * a;
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) T4[g][a * 4 + c] = Tm[a][c];
    }
  }
  __syncthreads();
  bool bad = false;
  const int jj = tid / LS_TPC, h = tid % LS_TPC;
  const unsigned gmask = 0xffu << (lane & ~(LS_TPC - 1));     // the eight lanes of this column
  for (int c0 = 0; c0 < n; c0 += LS_NC) {
    const int ncw = min(LS_NC, n - c0);
    for (int e0 = tid; e0 < l * ncw; e0 += 8 * LS_THREADS) {   // eight loads in flight per thread
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * LS_THREADS;
        x[u] = e < l * ncw ? xb[(int64_t)(e / ncw) * n + c0 + e % ncw] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * LS_THREADS;
        if (e < l * ncw) Cc[(e % ncw) * ldv + e / ncw] = ldexpf(x[u], sh);
      }
    }
    __syncthreads();
    const bool act = jj < ncw;
    float* x = Cc + jj * ldv;
    for (int g = 0; g < ng; ++g) {                        // x <- (H_t0 .. H_t0+3)^T x
      const int t0 = 4 * g;
      const float* v0 = V + t0 * ldv;
      const int i0 = t0 + ((h - t0 % LS_TPC) + LS_TPC) % LS_TPC;
      float w[4] = {0.f, 0.f, 0.f, 0.f};
      if (act)
        for (int i = i0; i < l; i += LS_TPC) {
          const float xi = x[i];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            // v_c(i) = 0 above its diagonal (V holds R there); columns past r are absent
            const float vc = (i < t0 + c || t0 + c >= r) ? 0.f : v0[c * ldv + i];
            w[c] = fmaf(vc, xi, w[c]);
          }
        }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = LS_TPC / 2; o > 0; o >>= 1) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
      float u[4];                                         // u = T_4^T w
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k <= c; ++k) a = fmaf(T4[g][k * 4 + c], w[k], a);
        u[c] = a;
      }
      if (act)
        for (int i = i0; i < l; i += LS_TPC) {
          float xi = x[i];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float vc = (i < t0 + c || t0 + c >= r) ? 0.f : v0[c * ldv + i];
            xi = fmaf(-u[c], vc, xi);
          }
          x[i] = xi;
        }
    }
    // z = R^{-1} (Q^T x)(0:r), column-oriented over the eight lanes of the column
    for (int q = r - 1; q >= 0; --q) {
      __syncwarp(gmask);                                  // row q of x is final
      const float z = act ? x[q] / rdiag[q] : 0.f;
      bad |= act && !isfinite(z);
      __syncwarp(gmask);                                  // every lane has read x[q]
      if (act) {
        if (h == q % LS_TPC) x[q] = z;
        for (int i = h; i < q; i += LS_TPC) x[i] = fmaf(-V[q * ldv + i], z, x[i]);
      }
    }
    __syncthreads();
    for (int e = tid; e < r * ncw; e += LS_THREADS) {
      const int q = e / ncw, c = e % ncw;
      zb[(int64_t)q * n + c0 + c] = (double)Cc[c * ldv + q];
    }
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += LS_THREADS) {         // the skeleton columns: unit vectors
    const int q = e / r, t = e % r;
    const int j = J[t];
    if (j >= 0 && j < n) zb[(int64_t)q * n + j] = q == t ? 1.0 : 0.0;
  }
  if (bad) record_error(p.dev_status, SKEL_ERR_NONFINITE, b);
}

}  // namespace
}  // namespace skel

using namespace skel;

struct skel_batch_plan {
  int nb = 0, kmax = 0, l = 0, lp = 0, stages = 0;
  double tol = 0.0;
  uint64_t seed = 0;
  int64_t mg = 0;                 // Gamma columns (max m_b rounded up to 32)
  BatchBlock* d_blocks = nullptr;
  CUtensorMap* d_tmaps = nullptr;
  SketchItem* d_items = nullptr;
  int n_items = 0;
  int32_t* d_order = nullptr;     // blocks grouped by cluster size
  int cls_count[3] = {0, 0, 0}, cls_off[3] = {0, 0, 0};
  size_t cls_smem[3] = {0, 0, 0};
  float* d_ghi = nullptr;
  float* d_glo = nullptr;
  CUtensorMap tm_ghi, tm_glo;
  float* d_X = nullptr;
  std::vector<int64_t> zoff;      // nb + 1 prefix offsets of Z (doubles)
  size_t sketch_smem = 0;
  int max_stages = 2;             // sketch pipeline depths that fit: 2 .. max_stages
  int concurrent = 0;             // LUPP cluster classes on parallel streams
  int32_t flags = 0;
  cudaStream_t cap = nullptr;     // capture / autotuning stream
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  cudaGraphExec_t exec = nullptr; // the captured run, bound to the outputs below
  const void* bound[4] = {nullptr, nullptr, nullptr, nullptr};
  int graph_launches = 0;
  // point plans (kernel blocks evaluated inside the sketch)
  bool points = false;
  int dim = 0;
  double inv_h2 = 0.0;
  float w_hi = 0.f, w_lo = 0.f;
  float* d_rec = nullptr;         // point records of every block
  PointSrc* d_src = nullptr;
  std::vector<int64_t> xoff;      // nb + 1 prefix offsets of X (floats)
};

namespace {

void plan_free(skel_batch_plan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  for (int i = 0; i < 2; ++i) {
    if (pl->side[i]) cudaStreamDestroy(pl->side[i]);
    if (pl->ev_join[i]) cudaEventDestroy(pl->ev_join[i]);
  }
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  cudaFree(pl->d_blocks);
  cudaFree(pl->d_tmaps);
  cudaFree(pl->d_items);
  cudaFree(pl->d_order);
  cudaFree(pl->d_ghi);
  cudaFree(pl->d_glo);
  cudaFree(pl->d_X);
  cudaFree(pl->d_rec);
  cudaFree(pl->d_src);
  delete pl;
}

size_t lupp_budget() {
  static size_t budget = 0;
  if (!budget) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, batch_lupp_kernel) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    budget = 227 * 1024 - fa.sharedSizeBytes - 256;
  }
  return budget;
}

size_t sketch_smem_for(int lp, int stages, bool pts) {
  return 1024 + (size_t)stages * (2 * (size_t)BS_ATILE + 2 * (size_t)lp * 128 + (pts ? BS_XREC : 0)) + 256;
}

// One run's launches on `st`: Gamma, the sketch, then the LUPP cluster classes, either one
// after the other on `st` or (plan->concurrent) class 0 on `st` and classes 1, 2 on the plan's
// side streams, forked from and joined back to `st`.  *launches: kernels enqueued.
skel_status enqueue_run(skel_batch_plan* pl, int32_t* Js, int32_t* ranks, double* Z, int32_t* dev_status,
                        cudaStream_t st, bool timers, int* launches) {
  int nl = 0;
  if (pl->points) {
    batch_points_prep_kernel<<<dim3(4, (unsigned)pl->nb), 256, 0, st>>>(pl->d_src, pl->dim, pl->inv_h2);
    ++nl;
  }
  batch_gamma_kernel<<<std::min<int64_t>(((int64_t)pl->lp * pl->mg / 4 + 255) / 256, 1024), 256, 0, st>>>(
      pl->l, pl->lp, pl->mg, (uint32_t)(pl->seed & 0xffffffffu), (uint32_t)(pl->seed >> 32), pl->d_ghi, pl->d_glo);
  ++nl;
  BatchSketchParams sp{};
  sp.blocks = pl->d_blocks;
  sp.tmaps = pl->d_tmaps;
  sp.items = pl->d_items;
  sp.X = pl->d_X;
  sp.l = pl->l;
  sp.lp = pl->lp;
  sp.stages = pl->stages;
  sp.scale = (float)(1.0 / std::sqrt((double)pl->l));
  sp.w_hi = pl->w_hi;
  sp.w_lo = pl->w_lo;
  sp.dev_status = dev_status;
  {
    KernelTimer kt(timers ? "batch_sketch" : nullptr, st);
    if (pl->points)
      batch_sketch_kernel<true><<<pl->n_items, BS_THREADS_P, pl->sketch_smem, st>>>(pl->tm_ghi, pl->tm_glo, sp);
    else
      batch_sketch_kernel<false><<<pl->n_items, BS_THREADS, pl->sketch_smem, st>>>(pl->tm_ghi, pl->tm_glo, sp);
  }
  ++nl;
  if (cudaGetLastError() != cudaSuccess) return SKEL_ERR_CUDA;
  BatchLuppParams lp{};
  lp.blocks = pl->d_blocks;
  lp.X = pl->d_X;
  lp.l = pl->l;
  lp.kmax = pl->kmax;
  lp.tol2 = (float)(pl->tol * pl->tol);
  lp.Js = Js;
  lp.ranks = ranks;
  lp.dev_status = dev_status;
  const bool fork = pl->concurrent && (pl->cls_count[1] > 0 || pl->cls_count[2] > 0);
  if (fork) {
    if (cudaEventRecord(pl->ev_fork, st) != cudaSuccess) return SKEL_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaStreamWaitEvent(pl->side[i], pl->ev_fork, 0) != cudaSuccess) return SKEL_ERR_CUDA;
  }
  // the side streams join `st` on every path out of here once they have been forked
  auto join = [&]() -> bool {
    bool ok = true;
    if (fork)
      for (int i = 0; i < 2; ++i)
        ok = cudaEventRecord(pl->ev_join[i], pl->side[i]) == cudaSuccess &&
             cudaStreamWaitEvent(st, pl->ev_join[i], 0) == cudaSuccess && ok;
    return ok;
  };
  for (int c = 0; c < 3; ++c) {
    if (pl->cls_count[c] == 0) continue;
    const int CL = 1 << c;
    cudaStream_t cs = fork && c > 0 ? pl->side[c - 1] : st;
    lp.order = pl->d_order + pl->cls_off[c];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(pl->cls_count[c] * CL));
    cfg.blockDim = dim3(BL_THREADS);
    cfg.dynamicSmemBytes = pl->cls_smem[c];
    cfg.stream = cs;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    {
      KernelTimer kt(timers ? "batch_lupp" : nullptr, cs);
      e = cudaLaunchKernelEx(&cfg, batch_lupp_kernel, lp);
    }
    ++nl;
    if (e != cudaSuccess) {
      join();
      return SKEL_ERR_CUDA;
    }
  }
  if (!join()) return SKEL_ERR_CUDA;
  BatchLsqParams zp{};
  zp.blocks = pl->d_blocks;
  zp.X = pl->d_X;
  zp.l = pl->l;
  zp.kmax = pl->kmax;
  zp.Js = Js;
  zp.ranks = ranks;
  zp.Z = Z;
  zp.dev_status = dev_status;
  {
    KernelTimer kt(timers ? "batch_z" : nullptr, st);
    batch_lsq_kernel<<<pl->nb, LS_THREADS, lsq_smem(pl->l, pl->kmax), st>>>(zp);
  }
  ++nl;
  if (cudaGetLastError() != cudaSuccess) return SKEL_ERR_CUDA;
  if (launches) *launches = nl;
  return SKEL_OK;
}

// Autotuning at plan creation: every pipeline depth of the sketch that fits and both
// schedules of the LUPP classes are run on the plan's own blocks (one warm-up, two timed runs
// each, CUDA events) and the fastest is kept.  Neither choice changes any result.
skel_status autotune(skel_batch_plan* pl) {
  int32_t *Js = nullptr, *ranks = nullptr, *st = nullptr;
  double* Z = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&Js, sizeof(int32_t) * (size_t)pl->nb * pl->kmax) == cudaSuccess &&
            cudaMalloc(&ranks, sizeof(int32_t) * (size_t)pl->nb) == cudaSuccess &&
            cudaMalloc(&st, 2 * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&Z, sizeof(double) * (size_t)std::max<int64_t>(pl->zoff[pl->nb], 1)) == cudaSuccess &&
            cudaMemset(st, 0, 2 * sizeof(int32_t)) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  float best = 1e30f;
  int best_stages = pl->stages, best_conc = 0;
  for (int stages = 2; ok && stages <= pl->max_stages; ++stages)
    for (int conc = 0; ok && conc < 2; ++conc) {
      pl->stages = stages;
      pl->sketch_smem = sketch_smem_for(pl->lp, stages, pl->points);
      pl->concurrent = conc;
      ok = enqueue_run(pl, Js, ranks, Z, st, pl->cap, false, nullptr) == SKEL_OK &&
           cudaEventRecord(e0, pl->cap) == cudaSuccess;
      for (int r = 0; ok && r < 2; ++r) ok = enqueue_run(pl, Js, ranks, Z, st, pl->cap, false, nullptr) == SKEL_OK;
      ok = ok && cudaEventRecord(e1, pl->cap) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (ok && ms < best) {
        best = ms;
        best_stages = stages;
        best_conc = conc;
      }
    }
  cudaStreamSynchronize(pl->cap);           // nothing of the trials is in flight past here
  int32_t hst[2] = {0, 0};
  if (ok) ok = cudaMemcpy(hst, st, sizeof(hst), cudaMemcpyDeviceToHost) == cudaSuccess;
  pl->stages = best_stages;
  pl->sketch_smem = sketch_smem_for(pl->lp, best_stages, pl->points);
  pl->concurrent = best_conc;
  cudaFree(Js);
  cudaFree(ranks);
  cudaFree(st);
  cudaFree(Z);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!ok) {
    cudaGetLastError();
    return SKEL_ERR_CUDA;
  }
  return hst[0] == 0 ? SKEL_OK : (skel_status)hst[0];
}

struct PointArgs {
  int dim;
  const float* const* x;
  const float* const* y;
  double h;
};

// Stored blocks (A, lda) or, with pts, Gaussian-kernel blocks given by point sets.
static skel_status plan_create(int32_t nblocks, const int64_t* m, const int64_t* n, const float* const* A,
                               const int64_t* lda, const PointArgs* pts, int32_t kmax, int32_t p, double tol,
                               uint64_t seed, int32_t flags, skel_batch_plan** plan) {
  if (plan == nullptr) return SKEL_ERR_INVALID_ARG;
  *plan = nullptr;
  if (nblocks < 1 || m == nullptr || n == nullptr) return SKEL_ERR_INVALID_ARG;
  if (pts == nullptr && (A == nullptr || lda == nullptr)) return SKEL_ERR_INVALID_ARG;
  if (pts && (pts->x == nullptr || pts->y == nullptr || pts->dim < 1 || pts->dim > 3 || !(pts->h > 0.0) ||
              !std::isfinite(pts->h) || !std::isfinite(1.0 / (pts->h * pts->h))))
    return SKEL_ERR_INVALID_ARG;
  if (kmax < 1 || kmax > BL_MAXK || p < 1 || kmax + p > BL_MAXL || !(tol >= 0.0) || !std::isfinite(tol))
    return SKEL_ERR_INVALID_ARG;
  if (flags & ~(SKEL_BATCH_GRAPH | SKEL_BATCH_AUTOTUNE)) return SKEL_ERR_INVALID_ARG;
  const int l = kmax + p, lp = (l + 15) / 16 * 16;
  const size_t budget = lupp_budget();
  if (budget == 0) return SKEL_ERR_CUDA;
  int64_t mmax = 0;
  std::vector<int> cls(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    if (m[b] < 1 || n[b] < 1 || m[b] > INT32_MAX || n[b] > INT32_MAX) return SKEL_ERR_INVALID_ARG;
    if (pts) {
      if (pts->x[b] == nullptr || pts->y[b] == nullptr) return SKEL_ERR_INVALID_ARG;
    } else {
      if (lda[b] < m[b] || A[b] == nullptr) return SKEL_ERR_INVALID_ARG;
      if (lda[b] % 4 != 0 || (reinterpret_cast<uintptr_t>(A[b]) & 15) != 0) return SKEL_ERR_UNSUPPORTED;
    }
    mmax = std::max(mmax, m[b]);
    int c = 0;
    while (c < 3 && lupp_smem(l, kmax, (int)((n[b] + (1 << c) - 1) >> c)) > budget) ++c;
    if (c == 3) return SKEL_ERR_UNSUPPORTED;       // wider than four CTAs' shared memory
    cls[b] = c;
  }
  EncodeTiledFn enc = encode_fn();
  if (!enc) return SKEL_ERR_UNSUPPORTED;
  int64_t npts = 0;
  if (pts)
    for (int b = 0; b < nblocks; ++b) npts += m[b] + n[b];
  skel_batch_plan* pl = new (std::nothrow) skel_batch_plan();
  if (!pl) return SKEL_ERR_WORKSPACE;
  pl->nb = nblocks;
  pl->kmax = kmax;
  pl->l = l;
  pl->lp = lp;
  pl->tol = tol;
  pl->seed = seed;
  pl->mg = (mmax + 31) / 32 * 32;
  pl->flags = flags;
  if (pts) {
    pl->points = true;
    pl->dim = pts->dim;
    pl->inv_h2 = 1.0 / (pts->h * pts->h);
    const double w = 2.0 * pl->inv_h2;
    pl->w_hi = (float)w;
    pl->w_lo = (float)(w - (double)pl->w_hi);
  }
  // shared memory of the sketch: 3 stages when they fit, else 2 (the autotuner may pick 2)
  pl->max_stages = sketch_smem_for(lp, 3, pts != nullptr) <= 227 * 1024 ? 3 : 2;
  pl->stages = pl->max_stages;
  pl->sketch_smem = sketch_smem_for(lp, pl->stages, pts != nullptr);

  std::vector<BatchBlock> hb(nblocks);
  std::vector<CUtensorMap> ht(pts ? 0 : nblocks);
  std::vector<SketchItem> items;
  std::vector<PointSrc> hsrc(pts ? nblocks : 0);
  // 32 records of padding: the last block's last 32-row step may copy past its x records
  if (pts && cudaMalloc(&pl->d_rec, sizeof(float) * kRec * (size_t)(npts + 32)) != cudaSuccess) {
    cudaGetLastError();
    plan_free(pl);
    return SKEL_ERR_CUDA;
  }
  pl->zoff.assign(nblocks + 1, 0);
  pl->xoff.assign(nblocks + 1, 0);
  int64_t xo = 0, ro = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (pts) {
      float* xr = pl->d_rec + ro * kRec;
      float* yr = xr + m[b] * kRec;
      ro += m[b] + n[b];
      hsrc[b] = PointSrc{pts->x[b], pts->y[b], (int32_t)m[b], (int32_t)n[b], xr, yr};
      hb[b] = BatchBlock{xr, 0, (int32_t)m[b], (int32_t)n[b], xo, pl->zoff[b], yr};
    } else {
      hb[b] = BatchBlock{A[b], lda[b], (int32_t)m[b], (int32_t)n[b], xo, pl->zoff[b], nullptr};
    }
    xo += (int64_t)l * n[b];
    pl->xoff[b + 1] = xo;
    pl->zoff[b + 1] = pl->zoff[b] + (int64_t)kmax * n[b];
    for (int t = 0; t < (int)((n[b] + 127) / 128); ++t) items.push_back(SketchItem{b, t});
    if (pts) continue;
    const cuuint64_t gdim[2] = {(cuuint64_t)m[b], (cuuint64_t)n[b]};
    const cuuint64_t gstride[1] = {(cuuint64_t)lda[b] * sizeof(float)};
    const cuuint32_t box[2] = {BS_BK, 128};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&ht[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A[b]), gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      plan_free(pl);
      return SKEL_ERR_UNSUPPORTED;
    }
  }
  // longest work first
  std::stable_sort(items.begin(), items.end(), [&](const SketchItem& a, const SketchItem& c) { return m[a.b] > m[c.b]; });
  pl->n_items = (int)items.size();
  std::vector<int32_t> order;
  for (int c = 0; c < 3; ++c) {
    pl->cls_off[c] = (int)order.size();
    std::vector<int32_t> v;
    for (int b = 0; b < nblocks; ++b)
      if (cls[b] == c) v.push_back(b);
    std::stable_sort(v.begin(), v.end(), [&](int a, int d) { return n[a] > n[d]; });
    for (int b : v) {
      order.push_back(b);
      pl->cls_smem[c] = std::max(pl->cls_smem[c], lupp_smem(l, kmax, (int)((n[b] + (1 << c) - 1) >> c)));
    }
    pl->cls_count[c] = (int)v.size();
  }
  bool ok = cudaMalloc(&pl->d_blocks, sizeof(BatchBlock) * nblocks) == cudaSuccess &&
            (pts || cudaMalloc(&pl->d_tmaps, sizeof(CUtensorMap) * nblocks) == cudaSuccess) &&
            (!pts || cudaMalloc(&pl->d_src, sizeof(PointSrc) * nblocks) == cudaSuccess) &&
            cudaMalloc(&pl->d_items, sizeof(SketchItem) * items.size()) == cudaSuccess &&
            cudaMalloc(&pl->d_order, sizeof(int32_t) * order.size()) == cudaSuccess &&
            cudaMalloc(&pl->d_ghi, sizeof(float) * (size_t)lp * pl->mg) == cudaSuccess &&
            cudaMalloc(&pl->d_glo, sizeof(float) * (size_t)lp * pl->mg) == cudaSuccess &&
            cudaMalloc(&pl->d_X, sizeof(float) * (size_t)std::max<int64_t>(xo, 1)) == cudaSuccess;
  ok = ok && cudaMemcpy(pl->d_blocks, hb.data(), sizeof(BatchBlock) * nblocks, cudaMemcpyHostToDevice) == cudaSuccess &&
       (pts || cudaMemcpy(pl->d_tmaps, ht.data(), sizeof(CUtensorMap) * nblocks, cudaMemcpyHostToDevice) ==
                   cudaSuccess) &&
       (!pts || cudaMemcpy(pl->d_src, hsrc.data(), sizeof(PointSrc) * nblocks, cudaMemcpyHostToDevice) == cudaSuccess) &&
       cudaMemcpy(pl->d_items, items.data(), sizeof(SketchItem) * items.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(pl->d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    const cuuint64_t gdim[2] = {(cuuint64_t)pl->mg, (cuuint64_t)lp};
    const cuuint64_t gstride[1] = {(cuuint64_t)pl->mg * sizeof(float)};
    const cuuint32_t box[2] = {BS_BK, (cuuint32_t)lp};
    const cuuint32_t es[2] = {1, 1};
    ok = enc(&pl->tm_ghi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl->d_ghi, gdim, gstride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
         enc(&pl->tm_glo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl->d_glo, gdim, gstride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  ok = ok && cudaFuncSetAttribute(batch_sketch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sketch_smem_for(lp, pl->max_stages, false)) == cudaSuccess &&
       cudaFuncSetAttribute(batch_sketch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sketch_smem_for(lp, pl->max_stages, true)) == cudaSuccess &&
       cudaFuncSetAttribute(batch_lupp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget) == cudaSuccess &&
       cudaFuncSetAttribute(batch_lsq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsq_smem(l, kmax)) ==
           cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < 2; ++i)
    ok = cudaStreamCreateWithFlags(&pl->side[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&pl->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    plan_free(pl);
    return SKEL_ERR_CUDA;
  }
  if (flags & SKEL_BATCH_AUTOTUNE) {
    const skel_status st = autotune(pl);
    if (st != SKEL_OK) {
      plan_free(pl);
      return st;
    }
  }
  *plan = pl;
  return SKEL_OK;
}

}  // namespace

extern "C" {

skel_status skel_batch_plan_create(int32_t nblocks, const int64_t* m, const int64_t* n, const float* const* A,
                                   const int64_t* lda, int32_t kmax, int32_t p, double tol, uint64_t seed,
                                   int32_t flags, skel_batch_plan** plan) {
  return plan_create(nblocks, m, n, A, lda, nullptr, kmax, p, tol, seed, flags, plan);
}

skel_status skel_batch_plan_create_points(int32_t nblocks, const int64_t* m, const int64_t* n, int32_t dim,
                                          const float* const* x, const float* const* y, double h, int32_t kmax,
                                          int32_t p, double tol, uint64_t seed, int32_t flags,
                                          skel_batch_plan** plan) {
  const PointArgs pa{dim, x, y, h};
  return plan_create(nblocks, m, n, nullptr, nullptr, &pa, kmax, p, tol, seed, flags, plan);
}

skel_status skel_batch_copy_sketch(const skel_batch_plan* plan, int32_t b, float* X, cudaStream_t stream) {
  if (plan == nullptr || X == nullptr || b < 0 || b >= plan->nb) return SKEL_ERR_INVALID_ARG;
  const int64_t cnt = plan->xoff[b + 1] - plan->xoff[b];
  if (cudaMemcpyAsync(X, plan->d_X + plan->xoff[b], sizeof(float) * (size_t)cnt, cudaMemcpyDeviceToDevice, stream) !=
      cudaSuccess)
    return SKEL_ERR_CUDA;
  return SKEL_OK;
}

skel_status skel_batch_z_offsets(const skel_batch_plan* plan, int64_t* offsets) {
  if (plan == nullptr || offsets == nullptr) return SKEL_ERR_INVALID_ARG;
  std::copy(plan->zoff.begin(), plan->zoff.end(), offsets);
  return SKEL_OK;
}

skel_status skel_batch_run(skel_batch_plan* plan, int32_t* Js, int32_t* ranks, double* Z, int32_t* dev_status,
                           cudaStream_t stream) {
  if (plan == nullptr || Js == nullptr || ranks == nullptr || Z == nullptr) return SKEL_ERR_INVALID_ARG;
  skel_batch_plan* pl = plan;
  if (!(pl->flags & SKEL_BATCH_GRAPH) || kernel_timing_enabled()) {
    int nl = 0;
    const skel_status st = enqueue_run(pl, Js, ranks, Z, dev_status, stream, true, &nl);
    note_launches(nl);
    return st;
  }
  const void* want[4] = {Js, ranks, Z, dev_status};
  if (pl->exec == nullptr || !std::equal(want, want + 4, pl->bound)) {
    // (re)capture the run bound to these outputs on the plan's stream
    if (pl->exec) {
      cudaGraphExecDestroy(pl->exec);
      pl->exec = nullptr;
    }
    if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SKEL_ERR_CUDA;
    int nl = 0;
    const skel_status st = enqueue_run(pl, Js, ranks, Z, dev_status, pl->cap, false, &nl);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(pl->cap, &g);
    if (st != SKEL_OK || ee != cudaSuccess || g == nullptr) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != SKEL_OK ? st : SKEL_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&pl->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      pl->exec = nullptr;
      cudaGetLastError();
      return SKEL_ERR_CUDA;
    }
    std::copy(want, want + 4, pl->bound);
    pl->graph_launches = nl;
  }
  if (cudaGraphLaunch(pl->exec, stream) != cudaSuccess) return SKEL_ERR_CUDA;
  note_launches(pl->graph_launches);
  return SKEL_OK;
}

skel_status skel_batch_plan_info(const skel_batch_plan* plan, int32_t* info) {
  if (plan == nullptr || info == nullptr) return SKEL_ERR_INVALID_ARG;
  info[0] = plan->stages;
  info[1] = plan->concurrent;
  info[2] = plan->flags;
  info[3] = plan->n_items;
  return SKEL_OK;
}

void skel_batch_plan_destroy(skel_batch_plan* plan) { plan_free(plan); }

}  // extern "C"
