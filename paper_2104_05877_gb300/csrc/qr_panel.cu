// Panel-blocked Householder QR of the tall skeleton C = A(:, Js) (m x s) on thread-block
// clusters, for the column ID Z = R_C^{-1} Q_C^T A (Eq. (2.1)) and the stable CUR of Remark 3.
//
// The s columns are factored in panels of b.  For a panel [t0, t0+b):
//   * PANEL (one cluster of CL CTAs; CTA k holds rows [k*mloc, (k+1)*mloc) of the panel
//     columns in shared memory, column-major).  Column c (global t = t0+c) is one step:
//       - every CTA holds the dot products of column c with the panel columns j >= c over its
//         rows >= t, and sends them (and the owner of row t sends row t) to every CTA with
//         st.async stores that complete on the receiver's mbarrier; each CTA sums the CL
//         partials in CTA order, so every CTA forms the same values:
//             D_j = x^T C(:, j),  sigma^2 = D_c,  alpha = C(t, c),  beta = -sign(alpha) sigma,
//             v = (x - beta e_t)/(alpha - beta),  tau = (beta - alpha)/beta,
//             w_j = v^T C(:, j) = (D_j - beta C(t, j))/(alpha - beta)       (j > c),
//             R(t, t0+j) = C(t, j) - tau w_j,  R(t, t) = beta;
//       - the CTA stores v, updates column c+1, then applies C(:, j) -= tau w_j v to the
//         columns j > c+1 while forming the next step's dot products in the same pass.
//     The panel kernel ends by writing V (explicit unit diagonal, zeros above).
//   * WY (grid-wide): G = V_p^T V_p by a split-K GEMM; with the compact WY form
//     Q_p = H_t0 .. H_t0+b-1 = I - V T V^T, T^{-1} = S = diag(G)/2 + strictly_upper(G), so
//     qr_wy_kernel forms V T^T and V T one row per thread by substitution with S.
//   * TRAIL (two grid-wide GEMMs): W = V^T C(t0:, t0+b:), C(t0:, t0+b:) -= (V T^T) W, which
//     applies Q_p^T to the columns to the right.  After the last panel, Q_C = Q_0 .. [I; 0]
//     from the panels' V T blocks, two GEMMs per panel.
// R entries above a panel (rows < t0 of its columns) are final when the panel is loaded and
// are written out from there.
#include <algorithm>

#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace skel {

namespace {

constexpr int kQrThreads = 512;
constexpr int kQrMaxB = 64;
constexpr int kQrInbox = 3;
constexpr size_t kQrSmemOptin = 227 * 1024;

template <typename T>
struct QrPanelParams {
  T* Cw; int64_t m, ldw;       // working copy of C (m x s, column-major)
  int s, t0, b, mloc;          // mloc: a multiple of 4
  T* V; int64_t ldv;           // out: reflectors, unit lower trapezoidal, m x s column-major
  T* VT;                       // out: V_p T_p^T, m x b column-major (ld = m)
  T* VTN;                      // out: V_p T_p in columns t0.. of an m x s column-major array
  double* R; int64_t ldr;      // out: s x s row-major
  int32_t* fail;
  int32_t* dev_status;
  GridComm gc;                 // grid panels: per-step slots of the CTAs' partial dot products
  T* growt;                    // grid panels: row t of the panel, [2][kQrMaxB]
};

__host__ __device__ constexpr int qr_b4(int b) { return (b + 3) / 4 * 4; }
// bytes one receiver takes in for step c: CL partial rows and the pivot row, columns
// 4*floor(c/4) .. b4-1 of each
template <typename T>
__host__ __device__ constexpr uint32_t qr_step_bytes(int CL, int b, int c) {
  return (uint32_t)(CL + 1) * (uint32_t)(qr_b4(b) - c / 4 * 4) * (uint32_t)sizeof(T);
}

template <typename T> __device__ __forceinline__ uint32_t qbits32(T v) { return __float_as_uint((float)v); }
template <typename T> __device__ __forceinline__ uint64_t qbits64(T v) { return (uint64_t)__double_as_longlong((double)v); }

// Send columns g0*4 .. b4-1 of src (shared memory) to dst_local (the same offset in every CTA
// of the cluster), 16 bytes per st.async; thread `slot` of `nslots` handles (receiver, group)
// pairs.
template <typename T>
__device__ __forceinline__ void qr_send(const T* src, uint32_t dst_local, uint32_t bar_local, int CL,
                                        int g0, int b4, int slot, int nslots) {
  const int groups = b4 / 4 - g0;
  for (int e = slot; e < CL * groups; e += nslots) {
    const int d = e / groups, g = g0 + e % groups;
    const uint32_t dst = map_cluster_u32(dst_local + (uint32_t)(g * 4 * sizeof(T)), d);
    const uint32_t bar = map_cluster_u32(bar_local, d);
    const T* v = src + 4 * g;
    if constexpr (sizeof(T) == 4) {
      st_async_v4_b32(dst, qbits32(v[0]), qbits32(v[1]), qbits32(v[2]), qbits32(v[3]), bar);
    } else {
      st_async_v2_b64(dst, qbits64(v[0]), qbits64(v[1]), bar);
      st_async_v2_b64(dst + 16, qbits64(v[2]), qbits64(v[3]), bar);
    }
  }
}

// The first n (<= 16) of 16 consecutive shared-memory elements into registers (zeros after
// them): 16-byte loads when aligned and n == 16.
template <typename T>
__device__ __forceinline__ void load16(const T* p, bool aligned, int n, T (&v)[16]) {
  if (aligned && n == 16) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 f = reinterpret_cast<const float4*>(p)[q];
        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double2 f = reinterpret_cast<const double2*>(p)[q];
        v[2 * q] = f.x; v[2 * q + 1] = f.y;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = k < n ? p[k] : T(0);
  }
}

// Four consecutive shared-memory elements (16-byte aligned for FP32, 8-byte for FP64).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

// Transposed butterfly reduction of NV per-lane values over the 32 lanes of a warp: halving
// levels (xor 16, 8, ...) each keep half of the values, so that afterwards lane l holds the
// warp totals of entries xr_index<NV>(l) + k, k < max(NV/32, 1); remaining levels sum fully.
template <int NV, typename T>
__device__ __forceinline__ void xreduce(T (&a)[NV], int lane) {
#pragma unroll
  for (int L = 0; L < 5; ++L) {
    const int m = 16 >> L;
    const int h = NV >> (L + 1);
    const bool up = (lane & m) != 0;
    if (h >= 1) {
#pragma unroll
      for (int k = 0; k < (NV >> (L + 1) > 0 ? NV >> (L + 1) : 1); ++k) {
        const T keep = up ? a[k + h] : a[k];
        const T send = up ? a[k] : a[k + h];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, m);
      }
    } else {
      a[0] += __shfl_xor_sync(0xffffffffu, a[0], m);
    }
  }
}
template <int NV>
__device__ __forceinline__ int xr_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int L = 0; L < 5; ++L) {
    const int h = NV >> (L + 1);
    if (h >= 1 && (lane & (16 >> L))) idx += h;
  }
  return idx;
}

constexpr int kQrMaxChunks = 8;       // rows per CTA <= 8 chunks of 512

// GRID: the panel is spread over a cooperative grid instead of one cluster (m too tall for a
// cluster's shared memory).  Each CTA then publishes its partial dot products (and the owner
// of row t that row) to a global slot per step, one grid barrier follows, and every CTA sums
// the G partials of each column itself in the same fixed order (lanes over CTAs, then a
// butterfly), so the reflector and every update are again identical in every CTA.
template <typename T, bool GRID>
__global__ void __launch_bounds__(kQrThreads, 1) qr_panel_kernel(const QrPanelParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = GRID ? (int)blockIdx.x : (int)cluster.block_rank();
  const int CL = GRID ? (int)gridDim.x : (int)cluster.num_blocks();
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  const int b = p.b, b4 = qr_b4(b), mloc = p.mloc, t0 = p.t0;
  const int64_t r0 = (int64_t)crank * mloc;
  const int ml = (int)(p.m - r0 < 0 ? 0 : (p.m - r0 < mloc ? p.m - r0 : mloc));

  __shared__ __align__(16) T part[GRID ? 1 : kQrInbox][GRID ? 1 : 16][kQrMaxB];   // partials per sender
  __shared__ __align__(16) T rowt[GRID ? 1 : kQrInbox][kQrMaxB];       // row t of the panel
  __shared__ __align__(8) uint64_t qbar[kQrInbox];
  __shared__ __align__(16) T dsum[kQrMaxB];                 // this step's summed dot products
  __shared__ __align__(16) T srow[kQrMaxB];                 // this step's row t
  __shared__ __align__(16) T wloc[kQrMaxB];                 // this CTA's partials for the next step
  __shared__ __align__(16) T rownext[kQrMaxB];              // row t+1 (owner)
  __shared__ T wv[kQrMaxB];                                 // tau * w_j of the current step
  __shared__ T wpart[4][kQrMaxB];                           // per-row-group partial dot products
  __shared__ int s_timeout, s_stop;
  T* P = reinterpret_cast<T*>(smem);                        // [b][mloc]

  if (*(volatile int32_t*)p.fail) return;
  if (tid == 0) {
    if constexpr (!GRID) {
      for (int k = 0; k < kQrInbox; ++k) mbar_init(smem_u32(&qbar[k]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    s_timeout = 0;
    s_stop = 0;
  }
  // grid panels: publish this CTA's partials (and row t, by its owner) for step c
  auto publish = [&](int c, bool owner) {
    if constexpr (GRID) {
      T* sl = reinterpret_cast<T*>(p.gc.slot(c, crank));
      for (int j = tid; j < b4; j += bd) sl[j] = wloc[j];
      if (owner)
        for (int j = tid; j < b4; j += bd) p.growt[(c & 1) * kQrMaxB + j] = rownext[j];
      comm_arrive(p.gc, c);
    }
  };
  // load the panel (rows past m are zero); rows above the panel hold final R entries
  for (int j0 = 0; j0 < b; j0 += 8)         // eight independent loads in flight per thread
    for (int i = tid; i < mloc; i += bd) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (j0 + u < b && i < ml) ? p.Cw[r0 + i + (int64_t)(t0 + j0 + u) * p.ldw] : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < b) {
          P[(size_t)(j0 + u) * mloc + i] = v[u];
          if (i < ml && r0 + i < t0) p.R[(r0 + i) * p.ldr + t0 + j0 + u] = (double)v[u];
        }
    }
  const uint32_t part0 = smem_u32(&part[0][0][0]), rowt0 = smem_u32(&rowt[0][0]), bar0 = smem_u32(&qbar[0]);
  auto part_dst = [&](int k) { return part0 + (uint32_t)(k * sizeof(part[0]) + crank * sizeof(part[0][0])); };
  auto rowt_dst = [&](int k) { return rowt0 + (uint32_t)(k * sizeof(rowt[0])); };
  auto bar_at = [&](int k) { return bar0 + (uint32_t)(k * sizeof(uint64_t)); };
  __syncthreads();

  // step 0's dot products: column 0 with every panel column over rows >= t0
  for (int j = warp; j < b4; j += nw) {
    T d = T(0);
    if (j < b)
      for (int i = lane; i < ml; i += 32)
        if (r0 + i >= t0) d = fma(P[i], P[(size_t)j * mloc + i], d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) wloc[j] = d;
  }
  const int owner0 = (int)(t0 / mloc);
  if (crank == owner0)
    for (int j = tid; j < b4; j += bd) rownext[j] = j < b ? P[(size_t)j * mloc + (t0 - r0)] : T(0);
  __syncthreads();
  if constexpr (GRID) {
    publish(0, crank == owner0);
  } else {
    if (tid == 0)
      for (int k = 0; k < kQrInbox && k < b; ++k) mbar_expect_tx(bar_at(k), qr_step_bytes<T>(CL, b, k));
    cluster.sync();     // barriers initialised and armed everywhere before the first send
    qr_send<T>(wloc, part_dst(0), bar_at(0), CL, 0, b4, tid, bd / 2);
    if (crank == owner0) qr_send<T>(rownext, rowt_dst(0), bar_at(0), CL, 0, b4, tid - bd / 2 >= 0 ? tid - bd / 2 : bd, bd / 2);
  }

  bool stopped = false;
  for (int c = 0; c < b; ++c) {
    const int64_t t = t0 + c;
    const int buf = c % kQrInbox;
    const uint32_t par = (uint32_t)((c / kQrInbox) & 1);
    if constexpr (GRID) {
      if (!comm_wait(p.gc, c, p.dev_status)) {       // uniform over the CTA
        if (tid == 0) atomicExch(p.fail, 1);
        stopped = true;
        break;
      }
      // dsum[j] = sum over the CTAs of their partials, in a fixed order (lanes over CTAs,
      // then a butterfly): the same bits in every CTA
      for (int j = (c & ~3) + warp; j < b4; j += nw) {
        T d = T(0);
        for (int k = lane; k < CL; k += 32) d += __ldcg(reinterpret_cast<const T*>(p.gc.slot(c, k)) + j);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) dsum[j] = d;
      }
      for (int j = tid; j < b4; j += bd) srow[j] = __ldcg(p.growt + (c & 1) * kQrMaxB + j);   // L2: slots are reused
    } else {
      if (warp == 0) {                   // one warp polls; the others wait at the CTA barrier
        const bool okw = mbar_wait(bar_at(buf), par, kDefaultWaitNs);
        if (!__all_sync(0xffffffffu, okw) && lane == 0 && atomicExch(&s_timeout, 1) == 0) {
          record_error(p.dev_status, SKEL_ERR_TIMEOUT, (int)t);
          atomicExch(p.fail, 1);
        }
      }
      __syncthreads();
      if (s_timeout) {
        stopped = true;
        break;
      }
      if (warp != 0) mbar_try_wait(bar_at(buf), par);   // acquire of the completed phase
      if (tid == bd - 1 && c + kQrInbox < b) mbar_expect_tx(bar_at(buf), qr_step_bytes<T>(CL, b, c + kQrInbox));
      // the partials of the CL CTAs summed in CTA order
      for (int j = tid; j < b4; j += bd) {
        T d = T(0);
        for (int k = 0; k < CL; ++k) d += part[buf][k][j];
        dsum[j] = d;
        srow[j] = rowt[buf][j];
      }
    }
    __syncthreads();
    // scalars of the reflector (every thread, same values)
    const T sig2 = dsum[c];
    const T alpha = srow[c];
    if (!isfinite(sig2) || sig2 == T(0)) {           // uniform over the cluster
      if (crank == 0 && tid == 0) {
        record_error(p.dev_status, isfinite(sig2) ? SKEL_ERR_RANK_DEFICIENT : SKEL_ERR_NONFINITE, (int)t);
        atomicExch(p.fail, 1);
      }
      stopped = true;
      break;
    }
    const T nrm = sqrt(sig2);
    const T beta = alpha != T(0) ? -copysign(nrm, alpha) : -nrm;
    const T den = alpha - beta;
    const T tau = (beta - alpha) / beta;
    // tau w_j and R(t, :) (threads over panel columns)
    if (tid < b) {
      const int j = tid;
      double rv = 0.0;
      if (j == c) {
        rv = (double)beta;
      } else if (j > c) {
        const T wj = (dsum[j] - beta * srow[j]) / den;
        wv[j] = tau * wj;
        rv = (double)(srow[j] - tau * wj);
      }
      if (crank == 0) p.R[t * p.ldr + t0 + j] = rv;
    }
    __syncthreads();
    const bool more = c + 1 < b;
    // reflector v (column c) and the update of column c+1 (x); threads over rows
    const T twn = more ? wv[c + 1] : T(0);
    const T rden = T(1) / den;
    for (int i = tid; i < ml; i += bd) {
      const int64_t gi = r0 + i;
      if (gi < t) continue;
      const T v = gi == t ? T(1) : P[(size_t)c * mloc + i] * rden;
      P[(size_t)c * mloc + i] = v;
      if (more) {
        const T x = fma(-twn, v, P[(size_t)(c + 1) * mloc + i]);
        P[(size_t)(c + 1) * mloc + i] = x;
        if (gi == t + 1) rownext[c + 1] = x;
      }
    }
    __syncthreads();
    if (!more) break;
    // columns j > c+1: C(:, j) -= tau w_j v; dot products of x with the columns j >= c+1 over
    // rows > t.  Warp (wr, wc): rows wr*128 .. +127 of every 512-row chunk (16 bytes per lane
    // per column), columns c+1+wc, c+1+wc+4, ...; eight columns at a time are reduced over
    // the lanes by a transposed butterfly into wpart[wr][j].  v and x are zero outside their
    // rows, so the update leaves the other rows unchanged.
    {
      const int wr = warp & 3, wc = warp >> 2;
      const int ncol = (b - (c + 1) - wc + 3) / 4;   // columns of this warp
      const int trel = (int)(t - r0);                // local index of row t (may be out of range)
      for (int q0 = 0; q0 < ncol; q0 += 8) {
        T pr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) pr[u] = T(0);
        for (int i0 = 0; i0 < mloc; i0 += 512) {
          const int ib = i0 + wr * 128 + 4 * lane;   // this lane's 4 rows
          if (ib >= mloc) continue;
          T vr[4], xr[4];
          ld4(P + c * mloc + ib, vr);
          ld4(P + (c + 1) * mloc + ib, xr);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (ib + e < trel) vr[e] = T(0);
            if (ib + e <= trel) xr[e] = T(0);
          }
          const int hit = trel + 1 - ib;             // 0..3: this lane holds row t+1
          int j = c + 1 + wc + 4 * q0;
          T* col = P + j * mloc + ib;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (q0 + u < ncol) {
              T y[4];
              ld4(col, y);
              if (j > c + 1) {
                const T f = -wv[j];
#pragma unroll
                for (int e = 0; e < 4; ++e) y[e] = fma(f, vr[e], y[e]);
                st4(col, y);
                if ((unsigned)hit < 4u) rownext[j] = hit == 0 ? y[0] : hit == 1 ? y[1] : hit == 2 ? y[2] : y[3];
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) pr[u] = fma(xr[e], y[e], pr[u]);
            }
            j += 4;
            col += 4 * mloc;
          }
        }
        xreduce<8>(pr, lane);
        const int q = q0 + xr_index<8>(lane);
        if ((lane & 3) == 0 && q < ncol) wpart[wr][c + 1 + wc + 4 * q] = pr[0];
      }
    }
    __syncthreads();
    if (tid < b4) {
      const int j = tid;
      T d = T(0);
      if (j >= c + 1 && j < b)
#pragma unroll
        for (int w = 0; w < 4; ++w) d += wpart[w][j];
      wloc[j] = d;
    }
    if (crank == (int)((t + 1) / mloc) && tid >= b && tid < b4) rownext[tid] = T(0);
    __syncthreads();
    const int own = (int)((t + 1) / mloc);
    if constexpr (GRID) {
      publish(c + 1, crank == own);
    } else {
      const int nb = (c + 1) % kQrInbox;
      const int g0 = (c + 1) / 4;
      qr_send<T>(wloc, part_dst(nb), bar_at(nb), CL, g0, b4, tid, bd / 2);
      if (crank == own) qr_send<T>(rownext, rowt_dst(nb), bar_at(nb), CL, g0, b4, tid - bd / 2 >= 0 ? tid - bd / 2 : bd, bd / 2);
    }
  }
  if (stopped && tid == 0) s_stop = 1;
  __syncthreads();
  const bool ok = !s_stop;              // uniform over the cluster (timeouts aside)
  // V_p (explicit unit diagonal, zeros above) back into P and out
  if (ok) {
    const int nq = mloc / 4;
    for (int e = tid; e < b * nq; e += bd) {
      const int k = e / nq, ib = 4 * (e % nq);
      const int kt = (int)(t0 + k - r0);             // local row of the diagonal of column k
      T v[4];
      ld4(P + k * mloc + ib, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = ib + u;
        v[u] = i >= ml ? T(0) : i > kt ? v[u] : (i == kt ? T(1) : T(0));
      }
      st4(P + k * mloc + ib, v);
      T* vout = p.V + r0 + ib + (int64_t)(t0 + k) * p.ldv;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ib + u < ml) vout[u] = v[u];
    }
  }
  __syncthreads();
  if constexpr (!GRID) cluster.sync();   // no CTA leaves while its peers may still address its shared memory
}

// V_p T_p^T (trailing update) and V_p T_p (formation of Q) for the rows t0.. of a panel, from
// V and G = V_p^T V_p (b x b, row-major), one row per thread across the grid.  With
// S = T_p^{-1} = diag(G)/2 + strictly_upper(G) (upper triangular):
//   (V T^T)(i, :) S^T = V(i, :):  z_j = (V_j - sum_{k>j} S(j, k) z_k) / S(j, j), j descending;
//   (V T)(i, :)   S   = V(i, :):  z_j = (V_j - sum_{k<j} z_k S(k, j)) / S(j, j), j ascending;
// in chunks of 16 columns held in registers, a solved chunk removed from the row in place.
constexpr int kWyRows = 128;

template <typename T>
size_t qr_wy_smem(int b) {
  return sizeof(T) * (2 * (size_t)b * b + kQrMaxB + 2 * (size_t)kWyRows * (b + 1));
}

template <typename T>
__global__ void __launch_bounds__(kWyRows) qr_wy_kernel(const T* V, int64_t ldv, int64_t m, int t0, int b,
                                                        const T* Gin, T* VT, T* VTN) {
  extern __shared__ __align__(16) unsigned char wsm[];
  constexpr int CH = 16;
  T* G = reinterpret_cast<T*>(wsm);                 // [b][b], upper triangle used
  T* GT = G + (size_t)b * b;                        // [b][b], GT[j][k] = G(k, j) for k <= j
  T* dinv = GT + (size_t)b * b;                     // [b]: 1 / S(j, j)
  T* rowA = dinv + kQrMaxB;                         // [kWyRows][b + 1]
  T* rowB = rowA + (size_t)kWyRows * (b + 1);
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += kWyRows) {
    const int r = e / b, j = e % b;
    const T g = j >= r ? Gin[e] : T(0);
    G[e] = g;
    GT[j * b + r] = g;
  }
  for (int j = tid; j < b; j += kWyRows) dinv[j] = T(2) / Gin[j * b + j];
  const int64_t i0 = t0 + (int64_t)blockIdx.x * kWyRows;
  for (int k = 0; k < b; ++k) {
    const int64_t i = i0 + tid;
    const T v = i < m ? V[i + (int64_t)(t0 + k) * ldv] : T(0);
    rowA[tid * (b + 1) + k] = v;
    rowB[tid * (b + 1) + k] = v;
  }
  __syncthreads();
  const int64_t i = i0 + tid;
  if (i >= m) return;
  const bool al = b % (16 / (int)sizeof(T)) == 0;  // 16-byte aligned rows of G and GT
  T* ra = rowA + tid * (b + 1);
  for (int h = (b - 1) / CH * CH; h >= 0; h -= CH) {
    const int nh = b - h < CH ? b - h : CH;
    T z[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) z[k] = k < nh ? ra[h + k] : T(0);
#pragma unroll
    for (int j = CH - 1; j >= 0; --j) {
      if (j < nh) {
        T col[16];                                   // S(h+k, h+j) = G(h+k, h+j), k < j
        load16(GT + (size_t)(h + j) * b + h, al, nh, col);
        z[j] *= dinv[h + j];
#pragma unroll
        for (int k = 0; k < j; ++k) z[k] = fma(-col[k], z[j], z[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k < nh) VT[i + (int64_t)(h + k) * m] = z[k];
    for (int j = 0; j < h; ++j) {
      T row[16];                                     // S(j, h+k) = G(j, h+k)
      load16(G + (size_t)j * b + h, al, nh, row);
      T y = ra[j];
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k < nh) y = fma(-row[k], z[k], y);
      ra[j] = y;
    }
  }
  T* rb = rowB + tid * (b + 1);
  for (int h = 0; h < b; h += CH) {
    const int nh = b - h < CH ? b - h : CH;
    T z[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) z[k] = k < nh ? rb[h + k] : T(0);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (j < nh) {
        T row[16];                                   // S(h+j, h+k) = G(h+j, h+k), k > j
        load16(G + (size_t)(h + j) * b + h, al, nh, row);
        z[j] *= dinv[h + j];
#pragma unroll
        for (int k = j + 1; k < CH; ++k)
          if (k < nh) z[k] = fma(-row[k], z[j], z[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k < nh) VTN[i + (int64_t)(t0 + h + k) * m] = z[k];
    for (int j = h + CH; j < b; ++j) {
      T col[16];                                     // S(h+k, j) = GT(j, h+k)
      load16(GT + (size_t)j * b + h, al, CH, col);
      T y = rb[j];
#pragma unroll
      for (int k = 0; k < CH; ++k) y = fma(-col[k], z[k], y);
      rb[j] = y;
    }
  }
}

struct QrPanelPlan {
  int CL = 0, b = 0, mloc = 0;   // CL: CTAs of the cluster, or of the cooperative grid when grid
  size_t smem = 0;
  bool grid = false;
};

template <typename T>
size_t qr_panel_smem(int b, int mloc) {
  return sizeof(T) * (size_t)b * mloc;
}

// Panels on one cooperative grid (one CTA per SM): G and the dynamic shared memory budget.
template <typename T>
void grid_panel_limits(int* G, size_t* budget) {
  static int g = -1;
  static size_t bud = 0;
  if (g < 0) {
    g = 0;
    cudaFuncAttributes fa{};
    int dev = 0, nsm = 0, per = 0;
    if (cudaFuncGetAttributes(&fa, qr_panel_kernel<T, true>) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      bud = kQrSmemOptin - fa.sharedSizeBytes - 1024;
      if (cudaFuncSetAttribute(qr_panel_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bud) ==
              cudaSuccess &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qr_panel_kernel<T, true>, kQrThreads, bud) == cudaSuccess &&
          per > 0)
        g = nsm;                          // one CTA per SM: the grid is co-resident
    }
    cudaGetLastError();
  }
  *G = g;
  *budget = bud;
}

// Matrices too tall for a cluster's shared memory: the panel rows spread over the grid, m/G
// rows per CTA, panels as wide as shared memory allows (32 columns at m = 262144).
template <typename T>
QrPanelPlan plan_qr_grid(int64_t m, int s) {
  QrPanelPlan pl;
  int G = 0;
  size_t budget = 0;
  grid_panel_limits<T>(&G, &budget);
  if (G < 2 || s < 1 || m < s) return pl;
  const int64_t mloc = ((m + G - 1) / G + 3) / 4 * 4;
  if (mloc > kQrMaxChunks * 512) return pl;
  int b = std::min(kQrMaxB, s);
  while (b >= 8 && qr_panel_smem<T>(b, (int)mloc) > budget) b -= 4;
  if (b < std::min(8, s) || qr_panel_smem<T>(b, (int)mloc) > budget) return pl;
  pl.CL = G;
  pl.b = b;
  pl.mloc = (int)mloc;
  pl.smem = qr_panel_smem<T>(b, (int)mloc);
  pl.grid = true;
  return pl;
}

template <typename T>
QrPanelPlan plan_qr_panels(int64_t m, int s) {
  QrPanelPlan pl;
  static int max_cluster = -1;
  static size_t budget = 0;
  if (max_cluster < 0) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, qr_panel_kernel<T, false>) != cudaSuccess) {
      cudaGetLastError();
      return pl;
    }
    budget = kQrSmemOptin - fa.sharedSizeBytes - 1024;
    max_cluster = 8;
    if (cudaFuncSetAttribute(qr_panel_kernel<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(qr_panel_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kQrThreads);
      cfg.dynamicSmemBytes = budget;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, qr_panel_kernel<T, false>, &cfg) == cudaSuccess && nclusters > 0)
        max_cluster = 16;
    }
    cudaGetLastError();
  }
  if (s < 1 || m < s) return pl;
  const int CL = max_cluster;
  const int64_t mloc = ((m + CL - 1) / CL + 3) / 4 * 4;
  if (mloc > kQrMaxChunks * 512) return plan_qr_grid<T>(m, s);   // keep the row loops short
  int b = std::min(kQrMaxB, s);
  while (b >= 8 && qr_panel_smem<T>(b, (int)mloc) > budget) b -= 4;
  if (b < std::min(8, s) || qr_panel_smem<T>(b, (int)mloc) > budget) return plan_qr_grid<T>(m, s);
  // a cluster panel this narrow means many panels, each with its WY factor and trailing
  // products: the grid's wider panels cost a grid barrier per column instead
  if (b < 16) {
    const QrPanelPlan g = plan_qr_grid<T>(m, s);
    if (g.b >= 2 * b) return g;
  }
  pl.CL = CL;
  pl.b = b;
  pl.mloc = (int)mloc;
  pl.smem = qr_panel_smem<T>(b, (int)mloc);
  return pl;
}

// workspace: fail word, Cw (m x s), VTN (m x s), VT (m x kQrMaxB), W (kQrMaxB x s), G (kQrMaxB^2),
// split-K scratch
// Tensor-core scratch of the FP32 panel products V_p^T (.) (3xTF32, gemm_tc.cu): for every
// panel start and the three widths used (V_p, the trailing columns, Q's s columns).
size_t qr_tc_ws(int64_t m, int s) { return gemm_tc_workspace_bound(m, std::max(s, kQrMaxB), kQrMaxB); }

// The FP32 panel products run on the tensor cores when every tile is TMA-addressable: Cw and
// V have leading dimension m, Q has ldq (rows t0.. start 16-byte aligned when these are
// multiples of 4; panel starts are multiples of 8).
bool qr_tc_ok(int64_t m, int64_t ldq) { return m % 4 == 0 && ldq % 4 == 0 && gemm_tc_usable(m, 1, 1, nullptr, m, nullptr, m); }

// grid panels' exchange: barrier header, [2][G][kQrMaxB] partials, [2][kQrMaxB] row t
template <typename T>
size_t qr_comm_ws(int G) {
  return comm_header_bytes(0) + align_up(sizeof(T) * 2 * (size_t)G * kQrMaxB) + align_up(sizeof(T) * 2 * kQrMaxB);
}

template <typename T>
size_t qr_panels_ws(int64_t m, int s, const QrPanelPlan& pl) {
  const bool f64 = sizeof(T) == 8;
  size_t kws = 0;                     // split-K scratch of W = V_p^T C(t0:, t0+b:), any width
  for (int ntr = 1; ntr <= s; ++ntr) kws = std::max(kws, gemm_workspace(kQrMaxB, ntr, m, f64));
  if (!f64 && m % 4 == 0) kws = std::max(kws, qr_tc_ws(m, s));
  return 256 + 2 * align_up(sizeof(T) * (size_t)m * s) + align_up(sizeof(T) * (size_t)m * kQrMaxB) +
         align_up(sizeof(T) * (size_t)kQrMaxB * s) + align_up(sizeof(T) * kQrMaxB * kQrMaxB) +
         (pl.grid ? qr_comm_ws<T>(pl.CL) : 0) + kws;
}

// Q = [I_s; 0] before the panels are applied (m x s, leading dimension ldq)
template <typename T>
__global__ void eye_kernel(int64_t m, int s, T* Q, int64_t ldq) {
  for (int c = blockIdx.y; c < s; c += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
      Q[i + (int64_t)c * ldq] = i == c ? T(1) : T(0);
}

template <typename T>
skel_status run_qr_panels_t(const QrPanelPlan& pl, const T* C, int64_t m, int64_t ldc, int s, T* V,
                            int64_t ldv, double* R, int64_t ldr, T* Q, int64_t ldq, void* ws,
                            int32_t* dev_status, cudaStream_t st) {
  const bool f64 = sizeof(T) == 8;
  char* base = static_cast<char*>(ws);
  int32_t* fail = reinterpret_cast<int32_t*>(base);
  base += 256;
  T* Cw = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)m * s);
  T* VTN = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)m * s);
  T* VT = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)m * kQrMaxB);
  T* Wt = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)kQrMaxB * s);
  T* Gp = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * kQrMaxB * kQrMaxB);
  char* comm = pl.grid ? base : nullptr;
  if (pl.grid) base += qr_comm_ws<T>(pl.CL);
  void* kws = base;
  if (cudaMemsetAsync(fail, 0, 4, st) != cudaSuccess) return SKEL_ERR_CUDA;
  if (cudaMemset2DAsync(R, sizeof(double) * ldr, 0, sizeof(double) * s, s, st) != cudaSuccess) return SKEL_ERR_CUDA;
  if (cudaMemcpy2DAsync(Cw, sizeof(T) * m, C, sizeof(T) * ldc, sizeof(T) * m, s, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return SKEL_ERR_CUDA;
  if (pl.grid) {
    if (cudaFuncSetAttribute(qr_panel_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
        cudaSuccess)
      return SKEL_ERR_CUDA;
  } else {
    if (cudaFuncSetAttribute(qr_panel_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
        cudaSuccess)
      return SKEL_ERR_CUDA;
    if (pl.CL > 8 &&
        cudaFuncSetAttribute(qr_panel_kernel<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      return SKEL_ERR_CUDA;
  }
  const skel_dtype dt = f64 ? SKEL_F64 : SKEL_F32;
  const bool tc = !f64 && qr_tc_ok(m, Q ? ldq : m) && (reinterpret_cast<uintptr_t>(Q) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(V) & 15) == 0 && ldv % 4 == 0;
  QrPanelParams<T> p{};
  p.Cw = Cw; p.m = m; p.ldw = m; p.s = s; p.mloc = pl.mloc;
  p.V = V; p.ldv = ldv; p.VT = VT; p.VTN = VTN; p.R = R; p.ldr = ldr; p.fail = fail; p.dev_status = dev_status;
  if (pl.grid) {
    p.gc.counter = reinterpret_cast<unsigned int*>(comm);
    p.gc.abort = reinterpret_cast<int32_t*>(comm + 4);
    p.gc.keys = nullptr;
    p.gc.payload = comm + comm_header_bytes(0);
    p.gc.slot_bytes = (int64_t)sizeof(T) * kQrMaxB;
    p.gc.G = pl.CL;
    p.gc.wait_ns = kDefaultWaitNs;
    p.growt = reinterpret_cast<T*>(comm + comm_header_bytes(0) + align_up(sizeof(T) * 2 * (size_t)pl.CL * kQrMaxB));
  }
  // G = V_p^T V_p over rows t0.. for the b reflectors starting at column t0, then (qr_wy_kernel)
  // V_p T_p^T into VT and V_p T_p into VTN(:, t0 : t0+b).
  auto wy = [&](int t0, int b) -> skel_status {
    const T* Vp = V + t0 + (int64_t)t0 * ldv;
    if (tc) {
      if (launch_gemm_tc_tn(m - t0, b, b, reinterpret_cast<const float*>(Vp), ldv, reinterpret_cast<const float*>(Vp),
                            ldv, reinterpret_cast<float*>(Gp), b, nullptr, kws, dev_status, st, "gemm_qr") != cudaSuccess)
        return SKEL_ERR_CUDA;
    } else {
      GemmArgs g{};
      g.M = b; g.N = b; g.K = m - t0;
      g.L = View{Vp, ldv, 1}; g.l_dt = dt;
      g.B = View{Vp, 1, ldv}; g.b_dt = dt;
      g.out = Gp; g.out_sr = b; g.out_sc = 1; g.out_dt = dt;
      g.alpha = 1.0;
      g.splitk_ws = kws;
      g.timer = "gemm_qr";
      if (launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, st) != cudaSuccess) return SKEL_ERR_CUDA;
    }
    const size_t wsm = qr_wy_smem<T>(b);
    if (cudaFuncSetAttribute(qr_wy_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm) != cudaSuccess)
      return SKEL_ERR_CUDA;
    KernelTimer kt("qr_wy", st);
    qr_wy_kernel<T><<<(unsigned)((m - t0 + kWyRows - 1) / kWyRows), kWyRows, wsm, st>>>(V, ldv, m, t0, b, Gp, VT, VTN);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
  };
  // Y (b x N, row-major, ld N) = V_p^T E(t0:, 0:N), then E(t0:, 0:N) -= L Y with L = the
  // (m - t0) x b block at Lm (leading dimension m): applies the block reflector to N columns.
  auto apply = [&](int t0, int b, const T* Lm, T* E, int64_t lde, int64_t N) -> skel_status {
    if (N <= 0) return SKEL_OK;
    const T* Vp = V + t0 + (int64_t)t0 * ldv;
    if (tc) {
      if (launch_gemm_tc_tn(m - t0, N, b, reinterpret_cast<const float*>(Vp), ldv, reinterpret_cast<const float*>(E),
                            lde, reinterpret_cast<float*>(Wt), N, nullptr, kws, dev_status, st, "gemm_qr") != cudaSuccess ||
          launch_rank_update_f32(m - t0, N, b, reinterpret_cast<const float*>(Lm), m, reinterpret_cast<const float*>(Wt),
                                 N, reinterpret_cast<float*>(E), lde, -1.0f, "gemm_qr", st) != cudaSuccess)
        return SKEL_ERR_CUDA;
      return SKEL_OK;
    }
    GemmArgs g{};
    g.M = b; g.N = N; g.K = m - t0;
    g.L = View{Vp, ldv, 1}; g.l_dt = dt;                // V_p^T(r, k) = V(t0+k, t0+r)
    g.B = View{E, 1, lde}; g.b_dt = dt;
    g.out = Wt; g.out_sr = N; g.out_sc = 1; g.out_dt = dt;
    g.alpha = 1.0;
    g.splitk_ws = kws;
    g.timer = "gemm_qr";
    if (launch_gemm(g, f64, LEFT_LOAD, EPI_STORE, st) != cudaSuccess) return SKEL_ERR_CUDA;
    GemmArgs h{};
    h.M = m - t0; h.N = N; h.K = b;
    h.L = View{Lm, 1, m}; h.l_dt = dt;
    h.B = View{Wt, N, 1}; h.b_dt = dt;
    h.out = E; h.out_sr = 1; h.out_sc = lde; h.out_dt = dt;
    h.alpha = -1.0;
    h.timer = "gemm_qr";
    return launch_gemm(h, f64, LEFT_LOAD, EPI_ACCUM, st) == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
  };
  // Super-panels of B columns (B a multiple of the cluster panel width b, at most kQrMaxB): a
  // panel updates only the later columns of its super-panel; at the end of the super-panel
  // its compact WY form (from V_B^T V_B) is applied once to every column to the right, and
  // Q_C is formed one super-panel at a time.  Where m is large the cluster's shared memory
  // limits b (12 columns at m = 65536), and B = 60 cuts the passes over the trailing columns
  // and over Q five-fold.
  const int B = pl.b * std::max(1, kQrMaxB / pl.b);
  for (int T0 = 0; T0 < s; T0 += B) {
    const int Bw = std::min(B, s - T0);
    for (int t0 = T0; t0 < T0 + Bw; t0 += pl.b) {
      p.t0 = t0;
      p.b = std::min(pl.b, T0 + Bw - t0);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(pl.CL);
      cfg.blockDim = dim3(kQrThreads);
      cfg.dynamicSmemBytes = qr_panel_smem<T>(p.b, pl.mloc);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      if (pl.grid) {
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
      } else {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = pl.CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
      }
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (pl.grid && cudaMemsetAsync(comm, 0, 256, st) != cudaSuccess) return SKEL_ERR_CUDA;   // barrier counter, abort
      {
        KernelTimer kt("qr_panel", st);
        const cudaError_t e = pl.grid ? cudaLaunchKernelEx(&cfg, qr_panel_kernel<T, true>, p)
                                      : cudaLaunchKernelEx(&cfg, qr_panel_kernel<T, false>, p);
        if (e != cudaSuccess) return SKEL_ERR_CUDA;
      }
      note_launches(1);
      const int nin = T0 + Bw - t0 - p.b;          // later columns of this super-panel
      if (nin > 0 || p.b == Bw) {
        const skel_status e = wy(t0, p.b);
        if (e != SKEL_OK) return e;
      }
      if (nin > 0) {
        const skel_status e = apply(t0, p.b, VT + t0, Cw + t0 + (int64_t)(t0 + p.b) * m, m, nin);
        if (e != SKEL_OK) return e;
      }
    }
    if (Bw > pl.b) {
      const skel_status e = wy(T0, Bw);
      if (e != SKEL_OK) return e;
    }
    const skel_status e = apply(T0, Bw, VT + T0, Cw + T0 + (int64_t)(T0 + Bw) * m, m, s - T0 - Bw);
    if (e != SKEL_OK) return e;
  }
  if (Q == nullptr) return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
  // Q_C = Q_0 Q_1 .. [I; 0] with Q_B = I - V_B T_B V_B^T per super-panel, applied from the last:
  // Y = V_B^T E(T0:, :), E(T0:, :) -= (V_B T_B) Y
  eye_kernel<T><<<dim3((unsigned)std::min<int64_t>((m + 255) / 256, 64), (unsigned)std::min(s, 1024)), 256, 0, st>>>(
      m, s, Q, ldq);
  note_launches(1);
  const int nsp = (s + B - 1) / B;
  for (int q = nsp - 1; q >= 0; --q) {
    const int T0 = q * B, Bw = std::min(B, s - T0);
    const skel_status e = apply(T0, Bw, VTN + T0 + (int64_t)T0 * m, Q + T0, ldq, s);
    if (e != SKEL_OK) return e;
  }
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

size_t qr_panels_workspace(skel_dtype dt, int64_t m, int32_t s) {
  if (dt == SKEL_F64) {
    const QrPanelPlan pl = plan_qr_panels<double>(m, s);
    return pl.b > 0 ? qr_panels_ws<double>(m, s, pl) : 0;
  }
  const QrPanelPlan pl = plan_qr_panels<float>(m, s);
  return pl.b > 0 ? qr_panels_ws<float>(m, s, pl) : 0;
}

skel_status run_qr_panels(skel_dtype dt, const void* C, int64_t m, int64_t ldc, int32_t s, void* V,
                          int64_t ldv, double* R, int64_t ldr, void* Q, int64_t ldq, void* ws, size_t ws_bytes,
                          int32_t* dev_status, cudaStream_t st) {
  if (dt == SKEL_F64) {
    const QrPanelPlan pl = plan_qr_panels<double>(m, s);
    if (pl.b == 0) return SKEL_ERR_UNSUPPORTED;
    if (ws_bytes < qr_panels_ws<double>(m, s, pl)) return SKEL_ERR_WORKSPACE;
    return run_qr_panels_t<double>(pl, (const double*)C, m, ldc, s, (double*)V, ldv, R, ldr, (double*)Q, ldq, ws,
                                   dev_status, st);
  }
  const QrPanelPlan pl = plan_qr_panels<float>(m, s);
  if (pl.b == 0) return SKEL_ERR_UNSUPPORTED;
  if (ws_bytes < qr_panels_ws<float>(m, s, pl)) return SKEL_ERR_WORKSPACE;
  return run_qr_panels_t<float>(pl, (const float*)C, m, ldc, s, (float*)V, ldv, R, ldr, (float*)Q, ldq, ws,
                                 dev_status, st);
}

}  // namespace skel
