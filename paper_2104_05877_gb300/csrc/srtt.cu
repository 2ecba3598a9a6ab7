// Subsampled randomized trigonometric transform (Sec. 2.3, item 2):
//     Gamma = sqrt(m/l) Pi_{m->l} T Phi Pi_{m->m},   T(k, r) = cas(2 pi k r / m) / sqrt(m),
// with (Pi_{m->m} a)_r = a_{pi(r)} and (Pi_{m->l} d)_i = d_{sel(i)}.  Entry by entry,
//     Gamma(i, q) = phi_r cas(2 pi sel(i) r / m) / sqrt(l),   r = pi^{-1}(q),
// so the tensor-core sketch regenerates Gamma's tiles from two small tables instead of a
// normal generator: tab[q] = pi^{-1}(q) | (phi < 0) << 31 (m words, padded to a multiple of
// 4 with zeros) and sel[i] (l words).  srtt_table_kernel forms both from the keyed Feistel
// permutations; srtt_dense_kernel writes Gamma (without the 1/sqrt(l)) for the SIMT GEMM.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

__global__ void srtt_table_kernel(uint32_t m, int32_t l, int64_t m4, int h, uint32_t k0, uint32_t k1,
                                  int32_t* tab, int32_t* sel) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < m4 + l; x += stride) {
    if (x < m) {
      const uint32_t r = (uint32_t)x;
      const uint32_t q = feistel_perm(r, m, h, k0, k1, kTagSrttPerm);
      const uint32_t neg = philox4x32_10(make_uint4(r, 0u, kTagSrttSign, 0u), k0, k1).x & 1u;
      if (q < m) tab[q] = (int32_t)(r | (neg << 31));     // always: the walk ends below m
    } else if (x < m4) {
      tab[x] = 0;
    } else {
      const int64_t i = x - m4;
      const uint32_t v = feistel_perm((uint32_t)i, m, h, k0, k1, kTagSrttSelect);
      sel[i] = (int32_t)(v < m ? v : 0u);
    }
  }
}

template <typename T>
__global__ void srtt_dense_kernel(uint32_t m, int32_t l, const int32_t* tab, const int32_t* sel, uint64_t minv,
                                  T* G, int64_t ldg) {
  const float two_over_m = 2.0f / (float)m;
  for (int i = blockIdx.y; i < l; i += gridDim.y) {
    const uint32_t s = (uint32_t)sel[i];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
      if constexpr (sizeof(T) == 8)
        G[(int64_t)i * ldg + q] = srtt_entry_f64(s, tab[q], m, minv);
      else
        G[(int64_t)i * ldg + q] = srtt_entry_f32(s, tab[q], m, minv, two_over_m);
    }
  }
}

}  // namespace

uint64_t srtt_minv(int64_t m) { return ~0ull / (uint64_t)m; }

size_t srtt_table_words(int64_t m) { return (size_t)((m + 3) / 4 * 4); }

cudaError_t launch_srtt_tables(int64_t m, int32_t l, uint64_t seed, int32_t* tab, int32_t* sel, cudaStream_t st) {
  if (m < 1 || m > (int64_t)INT32_MAX || l < 1 || l > m) return cudaErrorInvalidValue;
  const int64_t m4 = (int64_t)srtt_table_words(m);
  const int64_t total = m4 + l;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
  srtt_table_kernel<<<blocks, 256, 0, st>>>((uint32_t)m, l, m4, feistel_half_bits(m), (uint32_t)(seed & 0xffffffffu),
                                            (uint32_t)(seed >> 32), tab, sel);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_srtt_dense(int64_t m, int32_t l, const int32_t* tab, const int32_t* sel, skel_dtype dt, void* G,
                              int64_t ldg, cudaStream_t st) {
  const dim3 grid((unsigned)std::min<int64_t>((m + 255) / 256, 64), (unsigned)std::min(l, 1024));
  if (dt == SKEL_F64)
    srtt_dense_kernel<double><<<grid, 256, 0, st>>>((uint32_t)m, l, tab, sel, srtt_minv(m), (double*)G, ldg);
  else
    srtt_dense_kernel<float><<<grid, 256, 0, st>>>((uint32_t)m, l, tab, sel, srtt_minv(m), (float*)G, ldg);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel
