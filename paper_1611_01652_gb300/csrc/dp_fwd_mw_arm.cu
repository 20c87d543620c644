// Launcher of the four-warp rollout kernel k_forward_mw for the compiled arm topologies (3-7
// links; rows on chip, solver tape recorded).
#include "dp_steps.cuh"
#include "dp_kernels.h"

template <class Q>
static cudaError_t launch_forward_mw_q(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps,
                                       int rollout, cudaStream_t s) {
  const size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_forward_mw<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_forward_mw<Q><<<T.Bp / 32, 128, smem, s>>>(T, D, x0, t0, nsteps, rollout);
  return cudaGetLastError();
}
cudaError_t launch_forward_mw_arm(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps, int rollout,
                                  cudaStream_t s) {
  switch (T.topo_id) {
    case ArmTopo<3>::id: return launch_forward_mw_q<ArmTopo<3>>(T, D, x0, t0, nsteps, rollout, s);
    case ArmTopo<4>::id: return launch_forward_mw_q<ArmTopo<4>>(T, D, x0, t0, nsteps, rollout, s);
    case ArmTopo<5>::id: return launch_forward_mw_q<ArmTopo<5>>(T, D, x0, t0, nsteps, rollout, s);
    case ArmTopo<6>::id: return launch_forward_mw_q<ArmTopo<6>>(T, D, x0, t0, nsteps, rollout, s);
    case ArmTopo<7>::id: return launch_forward_mw_q<ArmTopo<7>>(T, D, x0, t0, nsteps, rollout, s);
    default: return cudaErrorInvalidValue;
  }
}
