// Tensor-core Gaussian sketch (tcgen05); placeholder until the kernel lands.
#include "internal.h"

namespace skel {

cudaError_t launch_sketch_tc(int64_t, int64_t, const float*, int64_t, int32_t, skel_prec, uint64_t,
                             float*, int64_t, int32_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace skel
