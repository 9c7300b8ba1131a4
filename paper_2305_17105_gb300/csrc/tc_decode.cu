// tcgen05 tensor-core forms (FP16 / FP8) of the decode and the fused
// forward+backward -- under construction.
#include "ntc_device.cuh"
#include "ntc_internal.h"

namespace ntc {

cudaError_t launch_decode_tc(const ntc_material&, const float*, int64_t, void*, int, int,
                             cudaStream_t, int) {
  return cudaErrorNotSupported;
}

cudaError_t launch_backward_tc(const ntc_material&, const BwdArgs&, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace ntc
