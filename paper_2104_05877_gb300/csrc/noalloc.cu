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

// The host-side name g_lupp_scratch is not a device address.  Its address in a context is
// looked up once, with that context current, and cached under the context's unique id: a
// device reset (which destroys the primary context and reloads the module, so the array may
// move) or a call from another context on the same device yields a new id and a new lookup.
constexpr int kCacheEntries = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  void* ptr;
};
ScratchEntry g_cache[kCacheEntries] = {};
int g_cache_next = 0;
std::mutex g_scratch_mu;

skel_status static_scratch(void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const unsigned long long id0 = current_context_id();
  if (id0 != 0)
    for (const ScratchEntry& e : g_cache)
      if (e.ctx_id == id0 && e.ptr != nullptr) {
        *out = e.ptr;
        return SKEL_OK;
      }
  // set-up for this context (the lookup also makes the current device's primary context
  // current when the thread has none)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_lupp_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SKEL_ERR_CUDA;
  }
  const unsigned long long id = current_context_id();
  if (id != 0) {        // without a context id every call looks the address up (no caching)
    g_cache[g_cache_next] = {id, p};
    g_cache_next = (g_cache_next + 1) % kCacheEntries;
  }
  *out = p;
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
