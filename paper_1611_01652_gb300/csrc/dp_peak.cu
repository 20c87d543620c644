// FP32 fused multiply-add throughput of the device, measured (not part of the method): the
// denominator of the roofline fraction of the FP32-bound kernels. Each thread runs
// DP_PEAK_CHAINS independent chains acc = acc * m + a, so the FMA pipe is never waiting on a
// dependency; the grid holds 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "../../include/dp.h"
#include "dp_world.h"

#define DP_PEAK_CHAINS 8

__global__ void __launch_bounds__(256) k_fma_peak(int64_t iters, float m, float a, float* out) {
  float acc[DP_PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < DP_PEAK_CHAINS; ++k) acc[k] = (float)(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < DP_PEAK_CHAINS; ++k) acc[k] = fmaf(acc[k], m, a);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < DP_PEAK_CHAINS; ++k) s += acc[k];
  if (s == 1.2345f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

extern "C" dp_status dp_fma_peak(int64_t iters, float* sink, int64_t* flops, void* stream) {
  if (iters < 1 || !sink || !flops) return dp_internal_fail(DP_EINVAL, "iters >= 1, sink and flops are required");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return dp_internal_fail(DP_ECUDA, "cannot query the device");
  const int blocks = 8 * sms, threads = 256;
  k_fma_peak<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, 0.999999f, 1e-7f, sink);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dp_internal_fail(DP_ECUDA, cudaGetErrorString(e));
  *flops = 2LL * blocks * threads * iters * 16 * DP_PEAK_CHAINS;
  return DP_OK;
}
