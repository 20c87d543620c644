// Launcher of the four-warp reverse-mode kernel k_backward_mw (compiled quadruped topology, whole
// solver tape).
#include "dp_steps.cuh"
#include "dp_kernels.h"

template <class Q>
static cudaError_t launch_backward_mw_q(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_backward_mw<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_backward_mw<Q><<<T.Bp / 32, 128, smem, s>>>(T, D);
  return cudaGetLastError();
}
cudaError_t launch_backward_mw_quadruped(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  return launch_backward_mw_q<QuadrupedTopo>(T, D, s);
}
