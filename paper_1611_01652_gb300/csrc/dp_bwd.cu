// Launchers of the one-warp reverse-mode kernel k_backward, and the choice between it and the
// four-warp kernel of dp_bwd_mw.cu.
#include "dp_steps.cuh"
#include "dp_kernels.h"

template <class Q>
static cudaError_t launch_backward_q(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_backward<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_backward<Q><<<T.Bp / 32, 32, smem, s>>>(T, D);
  return cudaGetLastError();
}
cudaError_t launch_backward(const DevTopo& T, const DevPtrs& D, cudaStream_t s) {
  // compiled topology with the whole tape: the solver's reverse sweeps on four warps per group
  if (T.topo_id != 0 && D.tape_full && !T.one_warp && !getenv("DP_SINGLE_WARP_BACKWARD"))
    return T.topo_id == QuadrupedTopo::id ? launch_backward_mw_quadruped(T, D, s) : launch_backward_mw_arm(T, D, s);
  if (T.topo_id == QuadrupedTopo::id) return launch_backward_q<QuadrupedTopo>(T, D, s);
  return launch_backward_q<DynTopo>(T, D, s);
}
