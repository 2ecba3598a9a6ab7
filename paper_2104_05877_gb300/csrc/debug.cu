// Test entry points for the generator: raw Philox words and the standard normals that the
// Gaussian sketch kernels generate (never stored by the sketch itself).
#include <curand_kernel.h>

#include "common.cuh"
#include "internal.h"

using namespace skel;

namespace {

__global__ void philox_kernel(const uint32_t* ctr, int64_t count, uint32_t k0, uint32_t k1, uint32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 o = philox4x32_10(c, k0, k1);
  out[4 * i] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
}

__global__ void gaussian_kernel(int32_t l, int64_t m, uint32_t k0, uint32_t k1, int as_fp64, void* G) {
  const int64_t m4 = (m + 3) / 4;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)l * m4) return;
  const uint32_t i = (uint32_t)(e / m4), j4 = (uint32_t)(e % m4);
  if (as_fp64) {
    double d[4];
    gaussian4_f64(k0, k1, i, j4, d);
    for (int q = 0; q < 4; ++q)
      if (4 * (int64_t)j4 + q < m) static_cast<double*>(G)[(int64_t)i * m + 4 * j4 + q] = d[q];
  } else {
    const float4 f = gaussian4_f32(k0, k1, i, j4);
    const float v[4] = {f.x, f.y, f.z, f.w};
    for (int q = 0; q < 4; ++q)
      if (4 * (int64_t)j4 + q < m) static_cast<float*>(G)[(int64_t)i * m + 4 * j4 + q] = v[q];
  }
}

// cuRAND's device Philox4_32_10 stream for (seed, subsequence = thread index), offset 0.
__global__ void curand_philox_kernel(uint64_t seed, int64_t nseq, int per_seq, uint32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseq) return;
  curandStatePhilox4_32_10_t stt;
  curand_init(seed, (unsigned long long)i, 0ull, &stt);
  for (int q = 0; q < per_seq; ++q) {
    const uint4 v = curand4(&stt);
    uint32_t* o = out + (i * per_seq + q) * 4;
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
}

// A grid-wide wait that can never complete: CTA `absent` does not publish step 0.  Every
// other CTA waits at most wait_ns and then reports SKEL_ERR_TIMEOUT.
__global__ void grid_wait_kernel(GridComm gc, int absent, int32_t* dev_status) {
  if ((int)blockIdx.x == absent) return;
  comm_arrive(gc, 0);
  comm_wait(gc, 0, dev_status);
}

}  // namespace

extern "C" {

skel_status skel_debug_curand_philox(uint64_t seed, int64_t nseq, int per_seq, uint32_t* out,
                                     cudaStream_t stream) {
  if (nseq < 1 || per_seq < 1 || out == nullptr) return SKEL_ERR_INVALID_ARG;
  curand_philox_kernel<<<(unsigned)((nseq + 127) / 128), 128, 0, stream>>>(seed, nseq, per_seq, out);
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

skel_status skel_debug_grid_timeout(int grid, uint64_t wait_ns, void* ws, size_t* ws_bytes,
                                    int32_t* dev_status, cudaStream_t stream) {
  if (grid < 2 || grid > 256 || ws_bytes == nullptr || wait_ns > 5000000000ull) return SKEL_ERR_INVALID_ARG;
  const size_t need = comm_header_bytes(1);
  if (ws == nullptr) { *ws_bytes = need; return SKEL_OK; }
  if (*ws_bytes < need) return SKEL_ERR_WORKSPACE;
  char* base = static_cast<char*>(ws);
  GridComm gc{};
  gc.counter = reinterpret_cast<unsigned int*>(base);
  gc.abort = reinterpret_cast<int32_t*>(base + 4);
  gc.keys = nullptr;
  gc.payload = nullptr;
  gc.slot_bytes = 0;
  gc.G = grid;
  gc.wait_ns = wait_ns;
  if (cudaMemsetAsync(base, 0, need, stream) != cudaSuccess) return SKEL_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grid_wait_kernel, gc, 0, dev_status) == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

skel_status skel_debug_philox(const uint32_t* counters, int64_t count, uint32_t k0, uint32_t k1,
                              uint32_t* out, cudaStream_t stream) {
  if (count < 0 || (count > 0 && (!counters || !out))) return SKEL_ERR_INVALID_ARG;
  if (count == 0) return SKEL_OK;
  philox_kernel<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(counters, count, k0, k1, out);
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

skel_status skel_debug_gaussian(int32_t l, int64_t m, uint64_t seed, int as_fp64, void* G,
                                cudaStream_t stream) {
  if (l < 1 || m < 1 || G == nullptr || m > 0xFFFFFFFFll) return SKEL_ERR_INVALID_ARG;
  const int64_t total = (int64_t)l * ((m + 3) / 4);
  gaussian_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
      l, m, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), as_fp64, G);
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // extern "C"
