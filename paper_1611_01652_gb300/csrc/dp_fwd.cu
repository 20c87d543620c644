// Launchers of the persistent rollout kernel k_forward (rows on chip or in global memory; with
// or without the solver tape).
#include "dp_steps.cuh"
#include "dp_kernels.h"

template <class RV, bool REC, class Q>
static cudaError_t launch_forward_t(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps,
                                    int rollout, cudaStream_t s) {
  const size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_forward<RV, REC, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_forward<RV, REC, Q><<<T.Bp / 32, 32, smem, s>>>(T, D, x0, t0, nsteps, rollout);
  return cudaGetLastError();
}
cudaError_t launch_forward(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps, int rollout,
                           int record, cudaStream_t s) {
  // the compiled-topology path keeps its rows on chip; otherwise the run-time path. Its recorded
  // rollouts run on four warps per group (not the harvest or gait noise, and not when the world
  // asks for one warp per group). The compiled arms have no one-warp kernels of their own: their
  // other launches take the run-time path.
  if (T.topo_id != 0 && T.sm_rows >= 0 && record && rollout && !D.harvest && !D.u_noise && !T.one_warp &&
      !getenv("DP_SINGLE_WARP_FORWARD"))
    return T.topo_id == QuadrupedTopo::id ? launch_forward_mw_quadruped(T, D, x0, t0, nsteps, rollout, s)
                                          : launch_forward_mw_arm(T, D, x0, t0, nsteps, rollout, s);
  if (T.topo_id == QuadrupedTopo::id && T.sm_rows >= 0)
    return record ? launch_forward_t<SL, true, QuadrupedTopo>(T, D, x0, t0, nsteps, rollout, s)
                  : launch_forward_t<SL, false, QuadrupedTopo>(T, D, x0, t0, nsteps, rollout, s);
  if (T.sm_rows >= 0)
    return record ? launch_forward_t<SL, true, DynTopo>(T, D, x0, t0, nsteps, rollout, s)
                  : launch_forward_t<SL, false, DynTopo>(T, D, x0, t0, nsteps, rollout, s);
  return record ? launch_forward_t<GL, true, DynTopo>(T, D, x0, t0, nsteps, rollout, s)
                : launch_forward_t<GL, false, DynTopo>(T, D, x0, t0, nsteps, rollout, s);
}
