// skel_pivot_lupp_static: the column-wise LUPP of skel_pivot_lupp for callers that cannot
// allocate device memory.  Its scratch (grid-barrier counter, per-step argmax keys, candidate
// slots, and the column slab when it does not fit in shared memory) lives in a fixed-size
// array in this library's device image instead of a caller-provided workspace.
#include <mutex>

#include "common.cuh"
#include "internal.h"

using namespace skel;

namespace {

// Scratch shared by every call on a device; held by each device that loads the library until
// the process exits.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_lupp_scratch[kStaticScratchBytes];

// The host-side name g_lupp_scratch is not a device address: each device's address is looked
// up once, with that device current, and cached here.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

skel_status static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SKEL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lupp_scratch) != cudaSuccess || p == nullptr) return SKEL_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SKEL_OK;
}

}  // namespace

extern "C" skel_status skel_pivot_lupp_static(skel_dtype dtype, const void* X, int64_t l, int64_t n,
                                              int64_t ldx, int32_t s, int32_t* Js, void* L,
                                              int64_t ldl, void* R, int64_t ldr,
                                              int32_t* dev_status, cudaStream_t stream) {
  if ((dtype != SKEL_F64 && dtype != SKEL_F32) || X == nullptr || Js == nullptr) return SKEL_ERR_INVALID_ARG;
  if (s < 1 || s > kMaxS || s > l || s > n || n > 0x7FFFFFFFll) return SKEL_ERR_INVALID_ARG;
  if (ldx < n || (L && ldl < s) || (R && ldr < n)) return SKEL_ERR_INVALID_ARG;
  if (lupp_workspace(dtype, n, s, nullptr) > kStaticScratchBytes) return SKEL_ERR_WORKSPACE;
  void* ws = nullptr;
  const skel_status st = static_scratch(&ws);
  if (st != SKEL_OK) return st;
  // run_lupp clears the barrier counter and argmax keys in the scratch before its launch
  return run_lupp(dtype, X, n, ldx, s, Js, L, ldl, R, ldr, ws, kStaticScratchBytes, dev_status, stream);
}
