// The fused training step over a batch of materials in one persistent
// launch (the kernel lives in tc_train.cuh; this unit instantiates its
// batched form).
#include "tc_train.cuh"

namespace ntc {

cudaError_t launch_train_tc_batched(const TrainBatchDev* dev, const ntc_material& first,
                                    int64_t total_tiles, int k_lay, int dx_lay, cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  if (pipelines_for(first, k_lay, dx_lay) == 0) return cudaErrorNotSupported;
  return launch_class<true>(first, BwdArgs{}, dev, total_tiles, k_lay, dx_lay, s);
}

}  // namespace ntc
