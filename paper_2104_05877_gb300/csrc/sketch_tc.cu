// Tensor-core Gaussian sketch X = Gamma A (Algorithm 2, sketch step; Table 1, T_s = O(nnz(A) l)) on
// sm_103a: tcgen05.mma with FP32 accumulators in tensor memory, A streamed by TMA, Gamma
// generated in shared memory by Philox-4x32-10 + Box-Muller and never written to global
// memory.  Operands are TF32 (kind::tf32: A read as stored, Gamma rounded to TF32) or BF16
// (kind::f16: both rounded to BF16 to nearest-even in shared memory); accumulation is FP32.
//
// Orientation: one CTA computes a 128-row block of X (MMA M = 128 rows of Gamma) for up to
// 512 columns of A (two N = 256 MMAs, 512 TMEM columns), over a K-range of rows of A.
//   MMA A operand = Gamma tile (128 x 32), K-major, generated;
//   MMA B operand = A tile (32 rows of A x 512 columns), K-major (A is column-major): for TF32
//                   the 128-byte-swizzled FP32 tile exactly as TMA lands it; for BF16 a copy
//                   converted into the 64-byte-swizzled BF16 layout.
// Generation is shared: the CJ CTAs of a thread-block cluster (1 x CJ x 1, CJ in {1, 2, 4, 8})
// work on the same 128 Gamma rows and K-steps for CJ different column tiles of A.  Each CTA
// generates 128/CJ rows of every Gamma tile and pushes them into its peers' shared memory
// with bulk copies (cp.async.bulk shared::cta -> shared::cluster) that complete their bytes
// on the peer's stage barrier, so a generated normal feeds CJ x 512 columns of A.  CTAs that
// share an A tile for different row blocks of X are launched adjacently so that the tile is
// read from HBM once and served from L2 to the others.  A K-split fills the machine (CTA z
// takes the K-steps z, z + P, ...); partial sums go to a workspace and a reduce kernel
// applies 1/sqrt(l).
//
// Warp roles: warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM allocator, warps 4..11
// Gamma generators (then warps 4..7 drain TMEM: warp w owns lanes 32*(w%4)..+31); for BF16
// warps 12..19 convert each FP32 A tile to BF16.  Stage hand-offs use mbarriers: full/empty
// for the FP32 A stages (TMA -> MMA or converters), the BF16 stages (converters -> MMA) and
// the Gamma stages: a Gamma stage is full when the local generators have arrived and the
// peers' bytes have landed, and empty when the MMAs of all CJ CTAs have consumed it (the
// MMA commit is multicast to the cluster).  Every wait is bounded; on timeout the CTA
// records SKEL_ERR_TIMEOUT, stops issuing work, waits (bounded) for what is in flight, and
// all CTAs of a cluster meet at a final cluster barrier before any of them frees TMEM and
// exits.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace skel {

namespace {

namespace cg = cooperative_groups;
using namespace tc;

constexpr int OP_TF32 = 0, OP_BF16 = 1;
constexpr int GEN_GAUSS = 0, GEN_SRTT = 1;

constexpr int TC_M = 128;
constexpr int TC_BK = 32;              // K elements per stage (one 128-byte FP32 row of A)
constexpr int TC_N = 512;              // columns of A per CTA (TMEM columns)
constexpr int TC_GEN_WARP0 = 4;
constexpr int TC_GEN_WARPS = 8;
constexpr int TC_CVT_WARP0 = 12;
constexpr int TC_CVT_WARPS = 8;
constexpr uint32_t A_BYTES = TC_N * 128;        // FP32 A stage: 64 KB
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

template <int OP>
struct SkCfg {
  static constexpr bool kBf16 = OP == OP_BF16;
  static constexpr int THREADS = kBf16 ? 32 * (TC_CVT_WARP0 + TC_CVT_WARPS) : 32 * TC_CVT_WARP0;
  static constexpr int GS = 4;                                  // Gamma stages
  static constexpr int AS = 2;                                  // FP32 A stages (TMA)
  static constexpr int BS = kBf16 ? 2 : 0;                      // BF16 A stages
  static constexpr uint32_t G_ROW = kBf16 ? 64 : 128;           // bytes per Gamma row per stage
  static constexpr uint32_t G_BYTES = TC_M * G_ROW;
  static constexpr uint32_t B_BYTES = kBf16 ? TC_N * 64 : 0;
  // barriers: full_a, empty_a [AS]; full_g, empty_g [GS]; full_b, empty_b [BS]; done
  static constexpr int NBAR = 2 * AS + 2 * GS + 2 * BS + 1;
  static constexpr size_t SMEM = 1024 + GS * G_BYTES + AS * A_BYTES + BS * B_BYTES + 256;
  static_assert(NBAR * 8 + 8 <= 256, "barrier area");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct TcParams {
  int64_t m, n;
  int l;
  int P;                  // K-split: CTA z takes the K-steps z, z + P, z + 2P, ...
  int64_t ksteps;         // K-steps of TC_BK rows over m
  int64_t grow0;          // Gamma column of row 0 of A (a multiple of 4)
  uint32_t k0s, k1s;      // Philox key
  float* out;             // X (P == 1) or partial buffers [P][l][n]
  int64_t ldo;
  int64_t part_stride;    // elements between partial buffers
  float scale;            // applied when P == 1
  int direct;             // P == 1
  int32_t* dev_status;
  const int32_t* srtt_tab;   // GEN_SRTT: pi^{-1}(q) | (phi < 0) << 31, padded to a multiple of 4
  const int32_t* srtt_sel;   // GEN_SRTT: the l selected rows
  uint64_t srtt_minv;        // floor((2^64 - 1) / m)
  float srtt_two_over_m;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);    // .x (low half) = lo
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int OP, int GEN>
__global__ void __launch_bounds__(SkCfg<OP>::THREADS, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap tmapA, const TcParams p) {
  using C = SkCfg<OP>;
  constexpr int GS = C::GS, AS = C::AS, BS = C::BS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* gbuf = smem;                                  // [GS][G_BYTES]
  unsigned char* abuf = gbuf + GS * C::G_BYTES;                // [AS][A_BYTES]  FP32, TMA
  unsigned char* bbuf = abuf + AS * A_BYTES;                   // [BS][B_BYTES]  BF16
  uint64_t* bars = reinterpret_cast<uint64_t*>(bbuf + BS * C::B_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + C::NBAR);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  cg::cluster_group cluster = cg::this_cluster();
  const int CJ = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lb = blockIdx.x;                         // 128-row block of X
  const int64_t j0 = (int64_t)blockIdx.y * TC_N;     // first column of A
  const int kz = blockIdx.z;
  const int nk = (int)((p.ksteps - kz + p.P - 1) / p.P);
  auto krow = [&](int it) { return ((int64_t)kz + (int64_t)it * p.P) * TC_BK; };   // first row of A

  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  auto full_a = [&](int s) { return bar(s); };
  auto empty_a = [&](int s) { return bar(AS + s); };
  auto full_g = [&](int s) { return bar(2 * AS + s); };
  auto empty_g = [&](int s) { return bar(2 * AS + GS + s); };
  auto full_b = [&](int s) { return bar(2 * AS + 2 * GS + s); };
  auto empty_b = [&](int s) { return bar(2 * AS + 2 * GS + BS + s); };
  const uint32_t done = bar(2 * AS + 2 * GS + 2 * BS);
  const uint32_t slice = (uint32_t)(TC_M / CJ) * C::G_ROW;     // bytes of one CTA's Gamma rows

  if (tid == 0) {
    for (int s = 0; s < AS; ++s) {
      mbar_init(full_a(s), 1);
      mbar_init(empty_a(s), C::kBf16 ? TC_CVT_WARPS : 1);
    }
    for (int s = 0; s < GS; ++s) {
      mbar_init(full_g(s), TC_GEN_WARPS);
      mbar_init(empty_g(s), CJ);
    }
    for (int s = 0; s < BS; ++s) {
      mbar_init(full_b(s), TC_CVT_WARPS);
      mbar_init(empty_b(s), 1);
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
  cluster.sync();        // every CTA's barriers are initialised before any remote arrive
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    if (atomicExch(abort_flag, 1) == 0) record_error(p.dev_status, SKEL_ERR_TIMEOUT, -2);
  };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % AS;
        const uint32_t ph = (uint32_t)(it / AS) & 1u;
        if (aborted()) break;
        if (it >= AS && !mbar_wait(empty_a(s), ph ^ 1u, TC_WAIT_NS)) { fail(); break; }
        mbar_expect_tx(full_a(s), A_BYTES);
        const int x = (int)krow(it);
        const uint32_t dst = smem_u32(abuf + s * A_BYTES);
        tma_load_2d(dst, &tmapA, x, (int)j0, full_a(s));
        tma_load_2d(dst + A_BYTES / 2, &tmapA, x, (int)(j0 + TC_N / 2), full_a(s));
        ++issued;
      }
      // drain: every issued load must have landed before the CTA may exit
      for (int it = std::max(0, issued - AS); it < issued; ++it) {
        if (!mbar_wait(full_a(it % AS), (uint32_t)(it / AS) & 1u, TC_WAIT_NS)) fail();
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int sa = it % AS, sg = it % GS, sb = BS ? it % BS : 0;
        const uint32_t pa = (uint32_t)(it / AS) & 1u, pg = (uint32_t)(it / GS) & 1u;
        const uint32_t pb = BS ? (uint32_t)(it / BS) & 1u : 0u;
        if (aborted()) break;
        const bool okb = C::kBf16 ? mbar_wait(full_b(sb), pb, TC_WAIT_NS) : mbar_wait(full_a(sa), pa, TC_WAIT_NS);
        if (!okb || !mbar_wait(full_g(sg), pg, TC_WAIT_NS)) { fail(); break; }
        tc_fence_after();
        const uint32_t ga = smem_u32(gbuf + sg * C::G_BYTES);
        if constexpr (C::kBf16) {
          const uint32_t idesc = idesc_bf16(TC_M, TC_N / 2);
          const uint32_t ba = smem_u32(bbuf + sb * C::B_BYTES);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {         // K = 16 per MMA, 32 bytes
            const uint64_t adesc = sw64_desc(ga + kk * 32);
            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
            mma_bf16(tmem, adesc, sw64_desc(ba + kk * 32), idesc, acc);
            mma_bf16(tmem + TC_N / 2, adesc, sw64_desc(ba + C::B_BYTES / 2 + kk * 32), idesc, acc);
          }
          mma_commit(empty_b(sb));
        } else {
          const uint32_t idesc = idesc_tf32(TC_M, TC_N / 2);
          const uint32_t aa = smem_u32(abuf + sa * A_BYTES);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 8; ++kk) {          // K = 8 per MMA, 32 bytes
            const uint64_t adesc = sw128_desc(ga + kk * 32);
            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
            mma_tf32(tmem, adesc, sw128_desc(aa + kk * 32), idesc, acc);
            mma_tf32(tmem + TC_N / 2, adesc, sw128_desc(aa + A_BYTES / 2 + kk * 32), idesc, acc);
          }
          mma_commit(empty_a(sa));
        }
        if (CJ > 1)
          mma_commit_multicast(empty_g(sg), (uint16_t)((1u << CJ) - 1u));
        else
          mma_commit(empty_g(sg));
      }
      mma_commit(done);
    }
  } else if (warp >= TC_GEN_WARP0 && warp < TC_GEN_WARP0 + TC_GEN_WARPS) {
    // ---------------- Gamma generators: this CTA's 128/CJ rows of every tile ----------------
    const int gt = tid - TC_GEN_WARP0 * 32;            // 0..255
    const int rows_per = TC_M / CJ, r0 = crank * rows_per;
    const int calls = rows_per * (TC_BK / 4);          // Philox calls per tile slice
    for (int it = 0; it < nk; ++it) {
      const int s = it % GS;
      const uint32_t ph = (uint32_t)(it / GS) & 1u;
      if (aborted()) break;
      if (it >= GS && !mbar_wait_cl(empty_g(s), ph ^ 1u, TC_WAIT_NS)) { fail(); break; }
      unsigned char* g = gbuf + s * C::G_BYTES;
      const int64_t kt = krow(it);
      // independent Philox calls per thread: 4, 2 or 1 (CJ = 1, 2, 4), unrolled for ILP
      auto gen_call = [&](int c) {
        const int i = r0 + (c >> 3), grp = c & 7;      // row of the tile, 4-column group
        const int64_t row = (int64_t)lb * TC_M + i;
        const int64_t k = kt + 4 * grp;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < p.l && k < p.m) {
          if constexpr (GEN == GEN_SRTT) {
            // the table is padded to a multiple of 4 words: k .. k+3 are in bounds
            const int4 t = __ldg(reinterpret_cast<const int4*>(p.srtt_tab + k));
            const uint32_t s = (uint32_t)__ldg(p.srtt_sel + row), mm = (uint32_t)p.m;
            v = make_float4(srtt_entry_f32(s, t.x, mm, p.srtt_minv, p.srtt_two_over_m),
                            srtt_entry_f32(s, t.y, mm, p.srtt_minv, p.srtt_two_over_m),
                            srtt_entry_f32(s, t.z, mm, p.srtt_minv, p.srtt_two_over_m),
                            srtt_entry_f32(s, t.w, mm, p.srtt_minv, p.srtt_two_over_m));
          } else {
            v = gaussian4_f32(p.k0s, p.k1s, (uint32_t)row, (uint32_t)((p.grow0 + k) >> 2));
          }
          if (k + 1 >= p.m) v.y = 0.f;
          if (k + 2 >= p.m) v.z = 0.f;
          if (k + 3 >= p.m) v.w = 0.f;
        }
        if constexpr (C::kBf16) {
          const uint32_t off = (uint32_t)(i * 64 + (((grp >> 1) ^ ((i >> 1) & 3)) << 4) + (grp & 1) * 8);
          *reinterpret_cast<uint2*>(g + off) = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
        } else {
          v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w);
          const uint32_t off = (uint32_t)(i * 128 + ((grp ^ (i & 7)) << 4));
          *reinterpret_cast<float4*>(g + off) = v;
        }
      };
      if (calls == 1024) {
#pragma unroll
        for (int q = 0; q < 4; ++q) gen_call(gt + 256 * q);
      } else if (calls == 512) {
#pragma unroll
        for (int q = 0; q < 2; ++q) gen_call(gt + 256 * q);
      } else if (gt < calls) {          // CJ = 8: 128 calls, warps 4 .. 7 of the generators idle
        gen_call(gt);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        // this warp's rows: r0 + 4 w + 32 q .. + 3 for each q, contiguous per q
        const int w = gt >> 5;
        for (int q = 0; q * 256 < calls; ++q) {
          if (4 * w + 32 * q >= rows_per) continue;                // rows outside this CTA's slice
          const uint32_t src = smem_u32(g) + (uint32_t)(r0 + 4 * w + 32 * q) * C::G_ROW;
          for (int pr = 0; pr < CJ; ++pr)
            if (pr != crank) bulk_copy_to_peer(src, 4 * C::G_ROW, full_g(s), pr);
        }
        if (w == 0 && CJ > 1)
          mbar_expect_tx(full_g(s), (uint32_t)(CJ - 1) * slice);   // the peers' rows of this stage
        else
          mbar_arrive(full_g(s));
      }
    }
  } else if (C::kBf16 && warp >= TC_CVT_WARP0) {
    // ---------------- converters: FP32 A tile (128-byte swizzle) -> BF16 (64-byte swizzle) ----
    const int ct = tid - TC_CVT_WARP0 * 32;            // 0..255
    for (int it = 0; it < nk; ++it) {
      if (aborted()) break;
      const int sa = it % AS, sb = BS ? it % BS : 0;
      const uint32_t pa = (uint32_t)(it / AS) & 1u, pb = BS ? (uint32_t)(it / BS) & 1u : 0u;
      if (!mbar_wait(full_a(sa), pa, TC_WAIT_NS) || (it >= BS && !mbar_wait(empty_b(sb), pb ^ 1u, TC_WAIT_NS))) {
        fail();
        break;
      }
      const unsigned char* a32 = abuf + sa * A_BYTES;
      unsigned char* b16 = bbuf + sb * C::B_BYTES;
#pragma unroll 4
      for (int q = 0; q < (TC_N * TC_BK / 8) / (32 * TC_CVT_WARPS); ++q) {
        const int c = ct + 32 * TC_CVT_WARPS * q;      // 16-byte BF16 chunk: column n, K 8kc..8kc+7
        const int n = c >> 2, kc = c & 3;
        const int h = n >> 8, nn = n & 255, r = nn & 7;
        const unsigned char* src = a32 + h * (A_BYTES / 2) + nn * 128;
        const float4 x0 = *reinterpret_cast<const float4*>(src + (((2 * kc) ^ r) << 4));
        const float4 x1 = *reinterpret_cast<const float4*>(src + (((2 * kc + 1) ^ r) << 4));
        const uint4 o = make_uint4(pack_bf16(x0.x, x0.y), pack_bf16(x0.z, x0.w), pack_bf16(x1.x, x1.y),
                                   pack_bf16(x1.z, x1.w));
        *reinterpret_cast<uint4*>(b16 + h * (C::B_BYTES / 2) + nn * 64 + ((kc ^ (r >> 1)) << 4)) = o;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(full_b(sb));
        mbar_arrive(empty_a(sa));
      }
    }
  }

  // ---------------- epilogue: TMEM -> X (warps 4..7) ----------------
  if (warp >= TC_GEN_WARP0 && warp < TC_GEN_WARP0 + 4) {
    const bool ok = mbar_wait(done, 0, TC_WAIT_NS);
    if (!ok) fail();
    tc_fence_after();
    if (ok && !aborted()) {
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
          if (jc + 32 <= p.n && ((p.ldo & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 15) == 0)) {
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
  cluster.sync();        // no CTA leaves while a peer may still read its shared memory
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
  int lblocks, jtiles, P, CJ;
};

// Resident clusters of CJ CTAs of the kernel (0 if that cluster shape cannot be launched).
template <int OP, int GEN>
int active_clusters(int CJ) {
  static int cache[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
  if (cache[CJ] >= 0) return cache[CJ];
  int nc = 0;
  if (cudaFuncSetAttribute(sketch_tc_kernel<OP, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SkCfg<OP>::SMEM) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, CJ, 1);
    cfg.blockDim = dim3(SkCfg<OP>::THREADS);
    cfg.dynamicSmemBytes = SkCfg<OP>::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CJ;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&nc, sketch_tc_kernel<OP, GEN>, &cfg) != cudaSuccess) nc = 0;
  }
  cudaGetLastError();
  cache[CJ] = nc;
  return nc;
}

template <int OP, int GEN>
TcPlan plan_tc(int64_t m, int64_t n, int l) {
  TcPlan pl{};
  pl.lblocks = (l + TC_M - 1) / TC_M;
  pl.jtiles = (int)((n + TC_N - 1) / TC_N);
  pl.CJ = 1;
  int slots = device_sm_count();
  // Clusters of 4 along the column tiles share each Gamma tile.  Clusters of 8 (supported by
  // the generator) halve the generation per flop but were measured slower at 65536 x 32768,
  // l = 1100 (TF32 7.7 -> 11.0 ms, BF16 9.6 -> 12.9 ms): every stage waits for all eight CTAs'
  // MMAs before it is refilled.
  for (int cj : {4, 2}) {
    if (pl.jtiles % cj != 0) continue;
    const int nc = active_clusters<OP, GEN>(cj);
    if (nc > 0) {
      pl.CJ = cj;
      slots = nc * cj;
      break;
    }
  }
  if (pl.CJ == 1) {
    const int nc = active_clusters<OP, GEN>(1);
    if (nc > 0) slots = nc;
  }
  const int64_t ksteps = (m + TC_BK - 1) / TC_BK;
  int P = std::max(1, slots / std::max(1, pl.lblocks * pl.jtiles));
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, ksteps / 8));   // keep >= 8 K-steps per CTA
  pl.P = std::min(P, 16);
  return pl;
}

template <int OP, int GEN>
cudaError_t launch_tc_op(int64_t row0, int64_t m, int64_t n, const float* A, int64_t lda, int32_t l, uint64_t seed,
                         float* X, int64_t ldx, void* ws, int32_t* dev_status, cudaStream_t st,
                         const int32_t* srtt_tab, const int32_t* srtt_sel) {
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
  const TcPlan pl = plan_tc<OP, GEN>(m, n, l);
  TcParams p{};
  p.m = m; p.n = n; p.l = l;
  p.P = pl.P;
  p.ksteps = (m + TC_BK - 1) / TC_BK;
  p.grow0 = row0;
  p.k0s = (uint32_t)(seed & 0xffffffffu);
  p.k1s = (uint32_t)(seed >> 32);
  p.direct = pl.P == 1;
  p.scale = (float)(1.0 / std::sqrt((double)l));
  p.out = p.direct ? X : static_cast<float*>(ws);
  p.ldo = p.direct ? ldx : n;
  p.part_stride = (int64_t)l * n;
  p.dev_status = dev_status;
  p.srtt_tab = srtt_tab;
  p.srtt_sel = srtt_sel;
  p.srtt_minv = srtt_minv(m);
  p.srtt_two_over_m = (float)(2.0 / (double)m);
  cudaError_t e = cudaFuncSetAttribute(sketch_tc_kernel<OP, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SkCfg<OP>::SMEM);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.lblocks, pl.jtiles, pl.P);
  cfg.blockDim = dim3(SkCfg<OP>::THREADS);
  cfg.dynamicSmemBytes = SkCfg<OP>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = pl.CJ;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  {
    KernelTimer kt("sketch_tc", st);
    e = cudaLaunchKernelEx(&cfg, sketch_tc_kernel<OP, GEN>, tmap, p);
  }
  note_launches(1);
  if (e != cudaSuccess || p.direct) return e;
  tc_reduce_kernel<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(l, 128)), 256, 0, st>>>(
      static_cast<const float*>(ws), pl.P, p.part_stride, l, n, X, ldx, p.scale, dev_status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

size_t sketch_tc_workspace(int64_t m, int64_t n, int32_t l, skel_prec prec, bool srtt) {
  const bool bf = prec == SKEL_PREC_BF16;
  const TcPlan pl = srtt ? (bf ? plan_tc<OP_BF16, GEN_SRTT>(m, n, l) : plan_tc<OP_TF32, GEN_SRTT>(m, n, l))
                         : (bf ? plan_tc<OP_BF16, GEN_GAUSS>(m, n, l) : plan_tc<OP_TF32, GEN_GAUSS>(m, n, l));
  return pl.P > 1 ? align_up(sizeof(float) * (size_t)pl.P * l * n) : 0;
}

cudaError_t launch_sketch_tc(int64_t row0, int64_t m, int64_t n, const float* A, int64_t lda, int32_t l,
                             skel_prec prec, uint64_t seed, float* X, int64_t ldx, void* ws,
                             int32_t* dev_status, cudaStream_t st, const int32_t* srtt_tab,
                             const int32_t* srtt_sel) {
  if (prec != SKEL_PREC_TF32 && prec != SKEL_PREC_BF16) return cudaErrorNotSupported;
  const bool srtt = srtt_tab != nullptr;
  if (srtt && (srtt_sel == nullptr || row0 != 0 || (reinterpret_cast<uintptr_t>(srtt_tab) & 15) != 0))
    return cudaErrorNotSupported;
  if (m < 1 || n < 1) return cudaErrorNotSupported;
  if ((lda % 4) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
  if (m > (int64_t)INT32_MAX || n > (int64_t)INT32_MAX) return cudaErrorNotSupported;
  if (srtt)
    return prec == SKEL_PREC_BF16
               ? launch_tc_op<OP_BF16, GEN_SRTT>(0, m, n, A, lda, l, seed, X, ldx, ws, dev_status, st, srtt_tab, srtt_sel)
               : launch_tc_op<OP_TF32, GEN_SRTT>(0, m, n, A, lda, l, seed, X, ldx, ws, dev_status, st, srtt_tab, srtt_sel);
  return prec == SKEL_PREC_BF16
             ? launch_tc_op<OP_BF16, GEN_GAUSS>(row0, m, n, A, lda, l, seed, X, ldx, ws, dev_status, st, nullptr, nullptr)
             : launch_tc_op<OP_TF32, GEN_GAUSS>(row0, m, n, A, lda, l, seed, X, ldx, ws, dev_status, st, nullptr, nullptr);
}

}  // namespace skel
