// Launcher of the four-warp rollout kernel k_forward_mw (compiled quadruped topology, rows on
// chip, solver tape recorded).
#include "dp_steps.cuh"
#include "dp_kernels.h"

cudaError_t launch_forward_mw_quadruped(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps,
                                        int rollout, cudaStream_t s) {
  const size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_forward_mw<QuadrupedTopo>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_forward_mw<QuadrupedTopo><<<T.Bp / 32, 128, smem, s>>>(T, D, x0, t0, nsteps, rollout);
  return cudaGetLastError();
}
