// Launcher of the per-step reverse kernel k_backward_ext (the wide controller's path).
#include "dp_steps.cuh"
#include "dp_kernels.h"

template <class Q>
static cudaError_t launch_backward_ext_q(const DevTopo& T, const DevPtrs& D, int t, cudaStream_t s) {
  size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_backward_ext<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_backward_ext<Q><<<T.Bp / 32, 32, smem, s>>>(T, D, t);
  return cudaGetLastError();
}
cudaError_t launch_backward_ext(const DevTopo& T, const DevPtrs& D, int t, cudaStream_t s) {
  if (T.topo_id == QuadrupedTopo::id) return launch_backward_ext_q<QuadrupedTopo>(T, D, t, s);
  return launch_backward_ext_q<DynTopo>(T, D, t, s);
}
