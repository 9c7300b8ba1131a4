// ntc_train_step_noalloc: the optimisation step for callers that may not
// allocate device memory.  Its scratch gradient is a fixed array in the
// library's own device image instead of a caller-provided buffer.
#include <mutex>

#include "ntc_internal.h"

namespace {

// Scratch gradient shared by every call on a device (each GPU that loads the
// library holds this array until the process exits).
__device__ __align__(256) float g_noalloc_grad[NTC_NOALLOC_MAX_PARAMS];

std::mutex g_setup_mutex;
float* g_grad_ptr[64] = {};  // device address of g_noalloc_grad, per device

}  // namespace

extern "C" int ntc_train_step_noalloc(const ntc_material* m, const ntc_trainer* tr,
                                      const ntc_target* t, int64_t batch, uint64_t seed,
                                      const float* uvl_or_null, float* loss_out, int32_t flags,
                                      void* stream) {
  if (!tr) return ntc::report_error(NTC_ERR_ARG, "trainer is NULL");
  // the gradient of a gradient-only step would land in the private array,
  // where the caller cannot read it and the next call clears it
  if (flags & NTC_FLAG_GRAD_ONLY)
    return ntc::report_error(NTC_ERR_ARG,
                             "NTC_FLAG_GRAD_ONLY: the allocation-free step keeps its gradient "
                             "private; use ntc_train_step with a caller-owned tr->grad");
  if (tr->n_params <= 0 || tr->n_params > (int64_t)NTC_NOALLOC_MAX_PARAMS)
    return ntc::report_error(NTC_ERR_SHAPE,
                             "n_params = %lld: the allocation-free step holds at most %lld "
                             "parameters (NTC_NOALLOC_MAX_PARAMS)",
                             (long long)tr->n_params, (long long)NTC_NOALLOC_MAX_PARAMS);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ntc::report_error(NTC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return ntc::report_error(NTC_ERR_UNSUPPORTED, "device index %d", dev);
  float* grad = nullptr;
  {
    // one-time set-up per device (with that device current): the host-side
    // name of the array is not a device address; ask the runtime for it
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_grad_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_grad);
      if (e != cudaSuccess)
        return ntc::report_error(NTC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_grad_ptr[dev] = static_cast<float*>(p);
    }
    grad = g_grad_ptr[dev];
  }
  ntc_trainer with_scratch = *tr;
  with_scratch.grad = grad;
  // every argument check of the step runs before anything is put on the
  // stream, so a refused call leaves the stream untouched
  const int st = ntc_train_step_check(m, &with_scratch, t, batch, seed, uvl_or_null, loss_out, flags);
  if (st != NTC_OK) return st;
  // the step needs a zero gradient on entry; the array keeps whatever the
  // previous call (of any material) left in it
  e = cudaMemsetAsync(grad, 0, (size_t)tr->n_params * sizeof(float), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return ntc::report_error(NTC_ERR_CUDA, "clear scratch: %s", cudaGetErrorString(e));
  return ntc_train_step(m, &with_scratch, t, batch, seed, uvl_or_null, loss_out, flags, stream);
}
