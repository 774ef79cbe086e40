// FP64 throughput probe: the measured denominator of the FP64-ALU roofline
// that the rollout and adjoint kernels are reported against.  Every thread
// runs eight independent fused multiply-add chains x <- x b + c (b < 1, so the
// values stay near c / (1 - b)); a launch performs
// blocks * threads * iters * 8 FMAs = 2 x that many FP64 flops.
#include <cuda_runtime.h>

#include "dmx.h"
#include "dmx_runtime.h"

namespace {

__global__ void k_dfma_peak(int iters, double b, double c, double* sink) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1e-9 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == -1.0) sink[0] = s;   // never true; keeps the chains live
}

}  // namespace

extern "C" dmx_status dmx_fp64_peak(int32_t blocks, int32_t threads, int32_t iters, double* sink, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !sink)
    return dmx_fail(DMX_ERR_INVALID, "dmx_fp64_peak: blocks >= 1, threads a multiple of 32 in [32, 1024], "
                                          "iters >= 1 and a device sink are required");
  k_dfma_peak<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999999, 1e-7, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, cudaGetErrorString(e));
  return DMX_OK;
}
