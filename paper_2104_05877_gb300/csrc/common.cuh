// Shared device utilities of libskel: the counter-based generator, Box-Muller transform,
// device error recording and a bounded grid-wide all-gather for persistent kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/skel.h"

namespace skel {

constexpr int kMaxS = 1024;            // largest pivot count / panel width handled
constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // grid-wide wait limit: 2 s

// ------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

constexpr uint32_t kTagGaussian = 0;
constexpr uint32_t kTagSparse = 1;
constexpr uint32_t kTagSrttPerm = 2;
constexpr uint32_t kTagSrttSelect = 3;
constexpr uint32_t kTagSrttSign = 4;

// ------------------------------------------------------------------------------------
// SRTT randomness (Sec. 2.3, item 2).  A keyed pseudo-random permutation of 0..m-1: a
// balanced 4-round Feistel network on 2h bits (Luby-Rackoff), 4^h >= m, round function =
// Philox word x of the counter (R, round, tag, 0) masked to h bits, mapped onto 0..m-1 by
// cycle walking (Black-Rogaway: re-apply the network until the value is below m; the cycle
// through x returns to x within 4^h applications, so the loop is bounded).
// ------------------------------------------------------------------------------------
__host__ __device__ inline int feistel_half_bits(int64_t m) {
  int h = 1;
  while ((int64_t)1 << (2 * h) < m) ++h;
  return h;
}

__host__ __device__ __forceinline__ uint32_t feistel_perm(uint32_t x, uint32_t m, int h, uint32_t k0, uint32_t k1,
                                                 uint32_t tag) {
  const uint32_t mask = (1u << h) - 1u;
  const uint64_t walks = (uint64_t)1 << (2 * h);
  uint32_t y = x;
  for (uint64_t w = 0; w <= walks; ++w) {
    uint32_t L = y >> h, R = y & mask;
#pragma unroll
    for (uint32_t rnd = 0; rnd < 4; ++rnd) {
      const uint32_t f = philox4x32_10(make_uint4(R, rnd, tag, 0u), k0, k1).x & mask;
      const uint32_t t = L ^ f;
      L = R;
      R = t;
    }
    y = (L << h) | R;
    if (y < m) break;
  }
  return y;
}

// (a * b) mod m for a, b < m < 2^31 by Barrett reduction with minv = floor((2^64 - 1) / m):
// the quotient estimate is low by at most one, so one correction suffices.
__device__ __forceinline__ uint32_t mulmod_barrett(uint32_t a, uint32_t b, uint32_t m, uint64_t minv) {
  const uint64_t prod = (uint64_t)a * b;
  const uint64_t q = __umul64hi(prod, minv);
  uint64_t r = prod - q * m;
  if (r >= m) r -= m;
  return (uint32_t)r;
}

// One SRTT entry without the 1/sqrt(l) scale: phi * cas(2 pi (sel * r mod m) / m), where the
// table word t = r | (phi < 0) << 31 holds r = pi^{-1}(q) for column q of Gamma.
__device__ __forceinline__ float srtt_entry_f32(uint32_t sel, int32_t t, uint32_t m, uint64_t minv,
                                                float two_over_m) {
  const uint32_t x = mulmod_barrett(sel, (uint32_t)t & 0x7fffffffu, m, minv);
  float sn, cs;
  sincospif((float)x * two_over_m, &sn, &cs);
  const float v = cs + sn;
  return t < 0 ? -v : v;
}
__device__ __forceinline__ double srtt_entry_f64(uint32_t sel, int32_t t, uint32_t m, uint64_t minv) {
  const uint32_t x = mulmod_barrett(sel, (uint32_t)t & 0x7fffffffu, m, minv);
  double sn, cs;
  sincospi(2.0 * (double)x / (double)m, &sn, &cs);
  const double v = cs + sn;
  return t < 0 ? -v : v;
}

// u = (2*(x >> 9) + 1) * 2^-24: exact in FP32, in [2^-24, 1 - 2^-24].
__device__ __forceinline__ float unit_open_f32(uint32_t x) {
  return __uint2float_rn(((x >> 9) << 1) | 1u) * 5.9604644775390625e-8f;
}
__device__ __forceinline__ double unit_open_f64(uint32_t x) {
  return (double)(((x >> 9) << 1) | 1u) * 5.9604644775390625e-8;
}

// Box-Muller: (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2).
__device__ __forceinline__ float2 box_muller_f32(uint32_t a, uint32_t b) {
  const float r = sqrtf(-2.0f * logf(unit_open_f32(a)));
  float s, c;
  sincospif(2.0f * unit_open_f32(b), &s, &c);
  return make_float2(r * c, r * s);
}
__device__ __forceinline__ double2 box_muller_f64(uint32_t a, uint32_t b) {
  const double r = sqrt(-2.0 * log(unit_open_f64(a)));
  double s, c;
  sincospi(2.0 * unit_open_f64(b), &s, &c);
  return make_double2(r * c, r * s);
}

// Standard normals G(i, 4*j4 .. 4*j4+3) of the Gaussian embedding (Gamma = G / sqrt(l)).
__device__ __forceinline__ float4 gaussian4_f32(uint32_t k0, uint32_t k1, uint32_t i, uint32_t j4) {
  const uint4 w = philox4x32_10(make_uint4(j4, i, kTagGaussian, 0u), k0, k1);
  const float2 p = box_muller_f32(w.x, w.y), q = box_muller_f32(w.z, w.w);
  return make_float4(p.x, p.y, q.x, q.y);
}
__device__ __forceinline__ void gaussian4_f64(uint32_t k0, uint32_t k1, uint32_t i, uint32_t j4,
                                              double out[4]) {
  const uint4 w = philox4x32_10(make_uint4(j4, i, kTagGaussian, 0u), k0, k1);
  const double2 p = box_muller_f64(w.x, w.y), q = box_muller_f64(w.z, w.w);
  out[0] = p.x; out[1] = p.y; out[2] = q.x; out[3] = q.y;
}

// ------------------------------------------------------------------------------------
// Device status: int32[2] = {first error code, step}.  Never traps.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void record_error(int32_t* st, int code, int step) {
  if (st == nullptr) return;
  if (atomicCAS(st, 0, code) == 0) atomicExch(st + 1, step);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------------------------------
// Grid-wide step synchronisation for persistent cooperative kernels.
//   * arrival: one release-ordered atomicAdd per CTA on a monotonic counter (zeroed by the
//     host before the launch); step t is complete when the counter reaches G*(t+1);
//   * waiting: a single thread per CTA polls the counter (acquire), so polling traffic is G
//     loads per round on one line instead of one per thread;
//   * payload: every CTA owns slot b of two parity buffers; a CTA arrives at step t+1 only
//     after it has read step t, so two buffers suffice.  Payloads are read with L2-only
//     loads (__ldcg) because the same addresses are rewritten two steps later;
//   * keys: one packed 64-bit word per step for argmax reductions by atomicMax (zeroed by
//     the host), (order-preserving magnitude bits << 32) | (0xFFFFFFFF - index), so the
//     largest magnitude wins and equal magnitudes go to the lowest index.
// Every wait is bounded (wait_ns); a CTA that gives up sets `abort`, which makes the others
// give up at their next poll.
// ------------------------------------------------------------------------------------
struct GridComm {
  unsigned int* counter;
  int32_t* abort;
  unsigned long long* keys;
  char* payload;
  int64_t slot_bytes;
  int G;
  uint64_t wait_ns;
  __device__ __forceinline__ char* slot(int step, int b) const {
    return payload + ((int64_t)(step & 1) * G + b) * slot_bytes;
  }
};

// Bytes of the header region of a GridComm workspace: counter, abort, keys[nsteps].
__host__ __device__ inline size_t comm_header_bytes(int nsteps) {
  return 256 + (((size_t)8 * (nsteps > 0 ? nsteps : 1) + 255) / 256) * 256;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrive at `step` (after this CTA's payload writes; contains a __syncthreads).
__device__ __forceinline__ void comm_arrive(const GridComm& gc, int step) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(gc.counter, 1u);
  }
}

// Wait until every CTA arrived at `step`.  Returns false (uniformly over the CTA) on timeout
// or abort; the caller then leaves.
__device__ __forceinline__ bool comm_wait(const GridComm& gc, int step, int32_t* dev_status) {
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    const unsigned int target = (unsigned int)gc.G * (unsigned int)(step + 1);
    int fail = 0;
    if ((int)(ld_acquire_u32(gc.counter) - target) < 0) {
      const uint64_t t0 = global_ns();
      uint32_t it = 0;
      while ((int)(ld_acquire_u32(gc.counter) - target) < 0) {
        if ((++it & 15u) == 0) {
          if (ld_relaxed_gpu(gc.abort) != 0) { fail = 1; break; }
          if (global_ns() - t0 > gc.wait_ns) {
            fail = 2;
            atomicExch(gc.abort, 1);
            record_error(dev_status, SKEL_ERR_TIMEOUT, step);
            break;
          }
        }
      }
    }
    s_fail = fail;
  }
  __syncthreads();
  const int f = s_fail;
  __syncthreads();
  return f == 0;
}

__device__ __forceinline__ unsigned long long pack_key(float mag, int64_t idx) {
  return ((unsigned long long)__float_as_uint(mag) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)idx);
}
__device__ __forceinline__ int64_t key_index(unsigned long long key) {
  return (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}

// Block-wide argmax of (key, index): larger key wins; equal keys -> smaller index.
template <typename T>
struct KeyIdx {
  T key;
  int64_t idx;
};

template <typename T>
__device__ __forceinline__ bool better(T ka, int64_t ia, T kb, int64_t ib) {
  return (ka > kb) || (ka == kb && ia < ib);
}

template <typename T>
__device__ __forceinline__ KeyIdx<T> block_argmax(T key, int64_t idx) {
  __shared__ T sk[32];
  __shared__ int64_t si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (better(k2, i2, key, idx)) { key = k2; idx = i2; }
  }
  __syncthreads();
  if (lane == 0) { sk[warp] = key; si[warp] = idx; }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
    key = lane < nw ? sk[lane] : sk[0];
    idx = lane < nw ? si[lane] : si[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T k2 = __shfl_xor_sync(0xffffffffu, key, o);
      const int64_t i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if (lane == 0) { sk[0] = key; si[0] = idx; }
  }
  __syncthreads();
  KeyIdx<T> r{sk[0], si[0]};
  __syncthreads();
  return r;
}

// Block-wide sum (deterministic order for a fixed block size).
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T sv[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sv[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
    v = lane < nw ? sv[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sv[0] = v;
  }
  __syncthreads();
  const T r = sv[0];
  __syncthreads();
  return r;
}

// Magnitude key for pivot searches: NaN and Inf rank above every finite value so that a
// non-finite entry in a pivot row is always selected and then reported.
template <typename T>
__device__ __forceinline__ T pivot_key(T v) {
  const T a = fabs(v);
  return isfinite(a) ? a : T(INFINITY);
}

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float dmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float dsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdiv_rn(a, b); }

// The LU updates x - a*b: FP64 rounds the product and the difference separately (the textbook
// sequence, so FP64 factors equal those of a plain FP64 restatement bit for bit); FP32 uses one
// fused multiply-add (one rounding, half the instructions).  Every FP32 LUPP kernel uses the
// same form, so the FP32 paths agree with each other bit for bit.
__device__ __forceinline__ double msub(double x, double a, double b) { return __dsub_rn(x, __dmul_rn(a, b)); }
__device__ __forceinline__ float msub(float x, float a, float b) { return __fmaf_rn(-a, b, x); }
// R's row x / p from q = rdiv_prep(p), formed once per step: FP64 divides (correctly rounded
// quotient), FP32 multiplies by the correctly rounded reciprocal.
__device__ __forceinline__ double rdiv_prep(double p) { return p; }
__device__ __forceinline__ float rdiv_prep(float p) { return __frcp_rn(p); }
__device__ __forceinline__ double rdiv(double x, double q) { return __ddiv_rn(x, q); }
__device__ __forceinline__ float rdiv(float x, float q) { return __fmul_rn(x, q); }

}  // namespace skel
