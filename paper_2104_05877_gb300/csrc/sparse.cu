// Sparse sign embedding (Sec. 2.3, item 3; Table 1: T_s = O(nnz(A) zeta)) and the sketch of a
// CSC matrix.
//
// Column j of Gamma holds zeta values +-1/sqrt(zeta) at distinct rows chosen by Floyd's
// sampling algorithm from Philox words (counter (j, 0, 1, c)); word 0 carries the signs.
// A pattern kernel writes the m x zeta (row | sign<<31) table once per call into the
// workspace (4*zeta bytes per row of A, L2-resident for the sizes used here); the scatter
// kernels then stream A once, each CTA accumulating a tile of 32 columns of X in shared
// memory with shared-memory atomics, and write X rows coalesced.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int CT = 32;       // columns of X per CTA (dense A)
constexpr int CT_CSC = 8;    // columns of X per CTA (CSC A): one per warp
constexpr int JCH = 256;     // rows of A per table chunk

// Pattern of rows row0 .. row0+m-1 of A (counters use the global row index).
__global__ void sparse_pattern_kernel(int64_t row0, int64_t m, int32_t l, int32_t zeta, uint32_t k0, uint32_t k1,
                                      int32_t* table) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  uint32_t w[32];
  const int nw = 1 + zeta;
  for (int c = 0; 4 * c < nw; ++c) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)(row0 + j), 0u, kTagSparse, (uint32_t)c), k0, k1);
    w[4 * c] = o.x;
    if (4 * c + 1 < 32) w[4 * c + 1] = o.y;
    if (4 * c + 2 < 32) w[4 * c + 2] = o.z;
    if (4 * c + 3 < 32) w[4 * c + 3] = o.w;
  }
  int32_t rows[31];
  for (int q = 0; q < zeta; ++q) {
    const uint32_t J = (uint32_t)(l - zeta + q);
    const uint32_t t = (uint32_t)(((uint64_t)w[1 + q] * (uint64_t)(J + 1)) >> 32);
    bool seen = false;
    for (int p = 0; p < q; ++p) seen |= (rows[p] == (int32_t)t);
    rows[q] = seen ? (int32_t)J : (int32_t)t;
    const uint32_t neg = (w[0] >> q) & 1u;
    table[j * zeta + q] = rows[q] | (int32_t)(neg << 31);
  }
}

template <typename T>
__device__ __forceinline__ void scatter(T* acc, int32_t code, int cc, T v) {
  const int row = code & 0x7fffffff;
  atomicAdd(&acc[row * CT + cc], code < 0 ? -v : v);
}

// Dense A (m x n col-major): CTA owns 32 columns of X.
template <typename T>
__global__ void __launch_bounds__(256) sparse_dense_kernel(int64_t m, int64_t n, const T* A, int64_t lda,
                                                           int32_t l, int32_t zeta,
                                                           const int32_t* table, T* X, int64_t ldx,
                                                           T scale, int32_t* dev_status) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* acc = reinterpret_cast<T*>(smem);                                   // [l][CT]
  int32_t* tab = reinterpret_cast<int32_t*>(smem + sizeof(T) * (size_t)l * CT);  // [JCH][zeta]
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * CT;
  const int nc = (int)std::min<int64_t>(CT, n - c0);
  for (int e = tid; e < l * CT; e += blockDim.x) acc[e] = T(0);
  for (int64_t j0 = 0; j0 < m; j0 += JCH) {
    const int nj = (int)std::min<int64_t>(JCH, m - j0);
    __syncthreads();
    for (int e = tid; e < nj * zeta; e += blockDim.x) tab[e] = table[j0 * zeta + e];
    __syncthreads();
    for (int cc = 0; cc < nc; ++cc) {
      const T* col = A + (c0 + cc) * lda + j0;
      for (int jj = tid; jj < nj; jj += blockDim.x) {
        const T v = col[jj];
        if (v == T(0)) continue;
        for (int q = 0; q < zeta; ++q) scatter(acc, tab[jj * zeta + q], cc, v);
      }
    }
  }
  __syncthreads();
  bool bad = false;
  for (int e = tid; e < l * CT; e += blockDim.x) {
    const int r = e / CT, cc = e % CT;
    if (cc < nc) {
      const T v = acc[e] * scale;
      bad |= !isfinite(v);
      X[(int64_t)r * ldx + c0 + cc] = v;
    }
  }
  if (bad) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
}

// CSC A: one warp per column at a time, lanes over that column's nonzeros.
__global__ void __launch_bounds__(256) sparse_csc_kernel(int64_t n, const int64_t* col_ptr,
                                                         const int32_t* row_idx, const float* val,
                                                         int32_t l, int32_t zeta,
                                                         const int32_t* table, float* X, int64_t ldx,
                                                         float scale, int32_t* dev_status) {
  // acc[cc * lda + r]: a column's l sums are contiguous (odd stride), so the lanes of a warp,
  // which work on one column, add into banks spread by their random rows
  extern __shared__ __align__(16) unsigned char smem[];
  float* acc = reinterpret_cast<float*>(smem);
  const int lda = l | 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * CT_CSC;
  const int nc = (int)std::min<int64_t>(CT_CSC, n - c0);
  for (int e = tid; e < lda * CT_CSC; e += blockDim.x) acc[e] = 0.f;
  __syncthreads();
  for (int cc = warp; cc < nc; cc += nwarps) {
    const int64_t b = col_ptr[c0 + cc], e_ = col_ptr[c0 + cc + 1];
    float* ac = acc + cc * lda;
    // four nonzeros per lane per round, their indices, values and (for zeta = 8) two 16-byte
    // table rows loaded before any add, so that each lane has several loads in flight
    for (int64_t k0 = b; k0 < e_; k0 += 128) {
      int64_t j[4];
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + lane + 32 * u;
        j[u] = k < e_ ? (int64_t)__ldg(row_idx + k) : -1;
        v[u] = k < e_ ? __ldg(val + k) : 0.f;
      }
      if (zeta == 8) {
        int4 t[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j[u] >= 0) {
            const int4* tj = reinterpret_cast<const int4*>(table + j[u] * 8);
            t[u][0] = __ldg(tj);
            t[u][1] = __ldg(tj + 1);
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j[u] >= 0) {
            const int32_t codes[8] = {t[u][0].x, t[u][0].y, t[u][0].z, t[u][0].w,
                                      t[u][1].x, t[u][1].y, t[u][1].z, t[u][1].w};
#pragma unroll
            for (int q = 0; q < 8; ++q) atomicAdd(&ac[codes[q] & 0x7fffffff], codes[q] < 0 ? -v[u] : v[u]);
          }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j[u] >= 0) {
            const int32_t* tj = table + j[u] * zeta;
            for (int q = 0; q < zeta; ++q) {
              const int32_t code = __ldg(tj + q);
              atomicAdd(&ac[code & 0x7fffffff], code < 0 ? -v[u] : v[u]);
            }
          }
      }
    }
  }
  __syncthreads();
  bool bad = false;
  for (int e = tid; e < l * CT_CSC; e += blockDim.x) {
    const int r = e / CT_CSC, cc = e % CT_CSC;
    if (cc < nc) {
      const float v = acc[cc * lda + r] * scale;
      bad |= !isfinite(v);
      X[(int64_t)r * ldx + c0 + cc] = v;
    }
  }
  if (bad) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
}

// Gaussian Gamma applied to a CSC A: every nonzero (j, v) adds v * G(:, j); lanes own rows of X.
__global__ void __launch_bounds__(256) gauss_csc_kernel(int64_t n, const int64_t* col_ptr,
                                                        const int32_t* row_idx, const float* val,
                                                        int32_t l, uint32_t k0, uint32_t k1,
                                                        float* X, int64_t ldx, float scale,
                                                        int32_t* dev_status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * nwarps + warp;
  if (c >= n) return;
  const int64_t b = col_ptr[c], e_ = col_ptr[c + 1];
  bool bad = false;
  for (int i0 = 0; i0 < l; i0 += 32) {
    const int i = i0 + lane;
    float acc = 0.f;
    if (i < l) {
      for (int64_t k = b; k < e_; ++k) {
        const uint32_t j = (uint32_t)row_idx[k];
        const float4 g = gaussian4_f32(k0, k1, (uint32_t)i, j >> 2);
        const float gj = (j & 3) == 0 ? g.x : (j & 3) == 1 ? g.y : (j & 3) == 2 ? g.z : g.w;
        acc = fmaf(val[k], gj, acc);
      }
      const float v = acc * scale;
      bad |= !isfinite(v);
      X[(int64_t)i * ldx + c] = v;
    }
  }
  if (bad) record_error(dev_status, SKEL_ERR_NONFINITE, -1);
}

}  // namespace

size_t sparse_pattern_bytes(int64_t m, int32_t zeta) { return align_up(sizeof(int32_t) * (size_t)m * zeta); }

cudaError_t launch_sparse_pattern(int64_t row0, int64_t m, int32_t l, int32_t zeta, uint64_t seed, int32_t* table,
                                  cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  sparse_pattern_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(
      row0, m, l, zeta, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), table);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sparse_sketch_dense(int64_t m, int64_t n, skel_dtype dt, const void* A,
                                       int64_t lda, int32_t l, int32_t zeta,
                                       const int32_t* table, void* X, int64_t ldx,
                                       int32_t* dev_status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + CT - 1) / CT);
  const size_t tabb = sizeof(int32_t) * JCH * zeta;
  if (dt == SKEL_F64) {
    const size_t smem = sizeof(double) * (size_t)l * CT + tabb;
    cudaError_t e = cudaFuncSetAttribute(sparse_dense_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparse_dense_kernel<double><<<grid, 256, smem, st>>>(m, n, (const double*)A, lda, l, zeta, table,
                                                         (double*)X, ldx, 1.0 / sqrt((double)zeta), dev_status);
  } else {
    const size_t smem = sizeof(float) * (size_t)l * CT + tabb;
    cudaError_t e = cudaFuncSetAttribute(sparse_dense_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparse_dense_kernel<float><<<grid, 256, smem, st>>>(m, n, (const float*)A, lda, l, zeta, table,
                                                        (float*)X, ldx, (float)(1.0 / sqrt((double)zeta)), dev_status);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sparse_sketch_csc(int64_t m, int64_t n, const int64_t* col_ptr,
                                     const int32_t* row_idx, const float* val, int32_t l,
                                     int32_t zeta, const int32_t* table, float* X, int64_t ldx,
                                     int32_t* dev_status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * (size_t)(l | 1) * CT_CSC;
  cudaError_t e = cudaFuncSetAttribute(sparse_csc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  {
    KernelTimer kt("sparse_csc", st);
    sparse_csc_kernel<<<(unsigned)((n + CT_CSC - 1) / CT_CSC), 256, smem, st>>>(
        n, col_ptr, row_idx, val, l, zeta, table, X, ldx, (float)(1.0 / sqrt((double)zeta)), dev_status);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gauss_sketch_csc(int64_t m, int64_t n, const int64_t* col_ptr,
                                    const int32_t* row_idx, const float* val, int32_t l,
                                    uint64_t seed, float* X, int64_t ldx, int32_t* dev_status,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gauss_csc_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(
      n, col_ptr, row_idx, val, l, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), X, ldx,
      (float)(1.0 / sqrt((double)l)), dev_status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
