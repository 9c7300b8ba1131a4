// The fused training step in the FP8-E4M3 form (the kernel lives in
// tc_train.cuh; this unit instantiates its FP8 forward).
#include "tc_train.cuh"

namespace ntc {

cudaError_t launch_train_tc_f8(const ntc_material& m, const BwdArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  return launch_class_f8(m, a, (a.n + kRows - 1) / kRows, s);
}

}  // namespace ntc
