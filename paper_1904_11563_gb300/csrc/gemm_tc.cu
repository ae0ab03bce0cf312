// a3 on the tensor cores (placeholder until the tcgen05 kernel lands).
#include "device_common.cuh"

namespace bpx {

cudaError_t launch_gemm_tc(const DevGraph&, const DevPlan&, const void*, const void*, const void*,
                           const void*, int, int, int, int, bool, float*, float*, int,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace bpx
