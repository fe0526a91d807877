// Diagnostics (not part of the operation): the sustained FP64 fused multiply-add rate of the
// device, so that the FP64-pipe roofline of the plain FP64 SU3_Bench kernel has a measured peak
// beside the one derived from unit counts and the clock.
//
// Every thread runs 8 independent FMA chains (enough to cover the FP64 pipe's latency) for a
// given number of steps; the chains' values stay bounded (x <- x * c + d with |c| < 1), and the
// kernel stores their sum so that the compiler keeps every FMA.
#include <cuda_runtime.h>

#include <string>

#include "su3_internal.h"

namespace su3 {

constexpr int kDfmaChains = 8;

__global__ void __launch_bounds__(256) su3_dfma_rate_kernel(double* out, int steps, double c, double d) {
  double x[kDfmaChains];
#pragma unroll
  for (int i = 0; i < kDfmaChains; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int i = 0; i < kDfmaChains; ++i) x[i] = fma(x[i], c, d);
  }
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < kDfmaChains; ++i) sum += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

su3_status measure_dfma_rate(int steps, double* out_dev, int grid, const LaunchCtx& ctx, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx.stream);
  if (e == cudaSuccess) {
    su3_dfma_rate_kernel<<<grid, 256, 0, ctx.stream>>>(out_dev, steps, 0.999999, 1e-7);
    e = cudaGetLastError();
    if (e == cudaSuccess) ++*ctx.launches;
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, ctx.stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    *ctx.err = std::string("FP64 rate measurement: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  return SU3_OK;
}

}  // namespace su3
