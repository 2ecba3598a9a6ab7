// Test entry points for the generator: raw Philox words and the standard normals that the
// Gaussian sketch kernels generate (never stored by the sketch itself); and measurement aids
// for the rooflines: the FMA rate of the FP64 / FP32 pipes, and the latency of one round of
// the two exchanges the pivoting and QR kernels are built on (a grid-wide barrier through
// global memory, and a candidate exchange between the CTAs of a thread-block cluster).
#include <cooperative_groups.h>
#include <curand_kernel.h>

#include "cluster.cuh"
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

// Eight independent FMA chains per thread; the sum goes to `sink` only under a condition no
// input meets, so the chains are kept.
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(int64_t iters, T* sink) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x) * T(1e-7) + T(i);
  const T b = T(0.999999), c = T(1e-6);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T sum = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) sum += a[i];
  if (sum == T(-1.2345)) sink[blockIdx.x] = sum;
}

// `steps` grid-wide barrier rounds (comm_arrive / comm_wait of the persistent kernels) over
// gridDim.x co-resident CTAs; CTA 0 records the time of rounds 1 .. steps-1.
__global__ void grid_rounds_kernel(GridComm gc, int steps, double* ns_per_step, int32_t* dev_status) {
  uint64_t t0 = 0;
  for (int r = 0; r < steps; ++r) {
    if (r == 1 && blockIdx.x == 0 && threadIdx.x == 0) t0 = global_ns();
    comm_arrive(gc, r);
    if (!comm_wait(gc, r, dev_status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && steps > 1)
    *ns_per_step = (double)(global_ns() - t0) / (double)(steps - 1);
}

// `steps` rounds of the cluster exchange: every CTA sends a 16-byte header and `col_words`
// 32-bit words to every CTA of the cluster with st.async stores that complete on the
// receiver's mbarrier (three rotating inboxes, as in the LUPP panel kernel), then waits for
// its own inbox; an inbox is armed again for round r+3 as soon as round r completes.  CTA 0
// records the time of rounds 1 .. steps-1.  Waits are bounded (SKEL_ERR_TIMEOUT).
constexpr int kXBufWords = 4 + 64;       // header + up to 64 column words per sender
__global__ void __launch_bounds__(128) cluster_rounds_kernel(int steps, int col_words, double* ns_per_step,
                                                             int32_t* dev_status) {
  namespace cg = cooperative_groups;
  __shared__ __align__(16) uint32_t inbox[3][16][kXBufWords];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ int s_fail;
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), crank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t bytes = (uint32_t)CL * 4u * (4u + (uint32_t)col_words);
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(smem_u32(&bar[k]), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < 3 && k < steps; ++k) mbar_expect_tx(smem_u32(&bar[k]), bytes);
  }
  __syncthreads();
  cluster.sync();
  uint64_t t0 = 0;
  for (int r = 0; r < steps; ++r) {
    if (r == 1 && crank == 0 && tid == 0) t0 = global_ns();
    const int k = r % 3;
    if (tid < 32) {
      // lane d sends the header to CTA d; lanes split the column words over the destinations
      const uint32_t base = smem_u32(&inbox[k][crank][0]);
      if (lane < CL)
        st_async_v4_b32(map_cluster_u32(base, lane), (uint32_t)r, (uint32_t)crank, 0u, 0u,
                        map_cluster_u32(smem_u32(&bar[k]), lane));
      for (int e = lane; e < CL * (col_words / 4); e += 32) {
        const int d = e / (col_words / 4), w = 4 * (e % (col_words / 4));
        st_async_v4_b32(map_cluster_u32(base + 16u + 4u * (uint32_t)w, d), (uint32_t)w, 0u, 0u, 0u,
                        map_cluster_u32(smem_u32(&bar[k]), d));
      }
    }
    if (tid == 0) {
      if (!mbar_wait(smem_u32(&bar[k]), (uint32_t)(r / 3) & 1u, 1000000000ull)) {
        record_error(dev_status, SKEL_ERR_TIMEOUT, r);
        s_fail = 1;
      } else if (r + 3 < steps) {
        mbar_expect_tx(smem_u32(&bar[k]), bytes);
      }
    }
    __syncthreads();
    if (s_fail) break;
  }
  if (crank == 0 && tid == 0 && !s_fail && steps > 1)
    *ns_per_step = (double)(global_ns() - t0) / (double)(steps - 1);
  // leave only after every CTA's last sends have landed (no st.async into an exited CTA):
  // the last round's inbox completion above covers the stores addressed to this CTA, and the
  // final cluster barrier keeps every CTA resident until all of them have seen theirs
  cluster.sync();
}

}  // namespace

extern "C" {

skel_status skel_debug_fma_rate(int fp64, int64_t iters, int64_t* flops, void* sink, cudaStream_t stream) {
  if (iters < 1 || flops == nullptr || sink == nullptr) return SKEL_ERR_INVALID_ARG;
  const int grid = device_sm_count() * 8;
  *flops = (int64_t)grid * 256 * iters * 8 * 2;
  if (fp64)
    fma_rate_kernel<double><<<grid, 256, 0, stream>>>(iters, static_cast<double*>(sink));
  else
    fma_rate_kernel<float><<<grid, 256, 0, stream>>>(iters, static_cast<float*>(sink));
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

skel_status skel_debug_exchange_latency(int kind, int ctas, int steps, int col_words, double* ns_per_step, void* ws,
                                        size_t* ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if ((kind != 0 && kind != 1) || steps < 2 || steps > 1000000 || ns_per_step == nullptr || ws_bytes == nullptr)
    return SKEL_ERR_INVALID_ARG;
  if (kind == 0) {
    if (ctas < 2 || ctas > device_sm_count()) return SKEL_ERR_INVALID_ARG;
    const size_t need = comm_header_bytes(1);
    if (ws == nullptr) { *ws_bytes = need; return SKEL_OK; }
    if (*ws_bytes < need) return SKEL_ERR_WORKSPACE;
    char* base = static_cast<char*>(ws);
    GridComm gc{};
    gc.counter = reinterpret_cast<unsigned int*>(base);
    gc.abort = reinterpret_cast<int32_t*>(base + 4);
    gc.G = ctas;
    gc.wait_ns = 1000000000ull;
    if (cudaMemsetAsync(base, 0, need, stream) != cudaSuccess) return SKEL_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, grid_rounds_kernel, gc, steps, ns_per_step, dev_status) == cudaSuccess
               ? SKEL_OK : SKEL_ERR_CUDA;
  }
  if ((ctas != 2 && ctas != 4 && ctas != 8 && ctas != 16) || col_words < 0 || col_words > 64 || col_words % 4)
    return SKEL_ERR_INVALID_ARG;
  if (ws == nullptr) { *ws_bytes = 0; return SKEL_OK; }
  if (ctas > 8 &&
      cudaFuncSetAttribute(cluster_rounds_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return SKEL_ERR_UNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(128);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_rounds_kernel, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return SKEL_ERR_UNSUPPORTED;
  }
  note_launches(1);
  return cudaLaunchKernelEx(&cfg, cluster_rounds_kernel, steps, col_words, ns_per_step, dev_status) == cudaSuccess
             ? SKEL_OK : SKEL_ERR_CUDA;
}

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
