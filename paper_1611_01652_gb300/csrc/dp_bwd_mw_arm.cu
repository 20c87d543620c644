// Launcher of the four-warp reverse-mode kernel k_backward_mw for the compiled arm topologies
// (3-7 links, whole solver tape); the 6- and 7-link kernels are built in dp_bwd_mw_arm2.cu so that
// the two translation units compile in parallel.
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
cudaError_t launch_backward_mw_arm_long(const DevTopo& T, const DevPtrs& D, cudaStream_t s);  // dp_bwd_mw_arm2.cu
cudaError_t launch_backward_mw_arm(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  switch (T.topo_id) {
    case ArmTopo<3>::id: return launch_backward_mw_q<ArmTopo<3>>(T, D, s);
    case ArmTopo<4>::id: return launch_backward_mw_q<ArmTopo<4>>(T, D, s);
    case ArmTopo<5>::id: return launch_backward_mw_q<ArmTopo<5>>(T, D, s);
    default: return launch_backward_mw_arm_long(T, D, s);
  }
}
