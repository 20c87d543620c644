// The four-warp reverse-mode kernels of the 6- and 7-link arms (a translation unit of their own
// so that the build compiles them in parallel with the shorter arms' kernels).
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
cudaError_t launch_backward_mw_arm_long(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  switch (T.topo_id) {
    case ArmTopo<6>::id: return launch_backward_mw_q<ArmTopo<6>>(T, D, s);
    case ArmTopo<7>::id: return launch_backward_mw_q<ArmTopo<7>>(T, D, s);
    default: return cudaErrorInvalidValue;
  }
}
