// FP32 CUDA-core throughput probe: the denominator of the FP32 decode and
// training forms' ALU roofline, measured on the device that runs them.
#include "ntc_internal.h"

namespace ntc {
namespace {

constexpr int kProbeChains = 16;  // independent FMA chains per thread (latency hidden)
constexpr int kProbeBlock = 256;

// Each thread advances kProbeChains independent chains x <- x * a + b for
// `iters` rounds (2 flops per FMA); the sum is stored only if it equals a
// value it cannot take, so the chains are kept but nothing is written.
__global__ void __launch_bounds__(kProbeBlock) fma_probe_kernel(float* sink, int iters, float a,
                                                                 float b) {
  float x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  if (s == -1.2345e30f) sink[threadIdx.x] = s;
}

}  // namespace

cudaError_t probe_fma_tflops(float* tflops, cudaStream_t s) {
  const int blocks = sm_count() * 8, iters = 1 << 14;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    fma_probe_kernel<<<blocks, kProbeBlock, 0, s>>>(nullptr, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flop = 2.0 * kProbeChains * (double)iters * blocks * kProbeBlock;
    if (e == cudaSuccess && rep > 0 && ms > 0.f) {  // rep 0 warms up
      const float t = (float)(flop / (ms * 1e-3) / 1e12);
      best = t > best ? t : best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return e;
}

}  // namespace ntc
