// Launchers of the per-step reverse kernels of the wide controller's path: k_backward_ext (one
// warp per group of 32 instances) and k_backward_ext_mw (four warps per group: the compiled
// topology with the whole tape).
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
template <class Q>
static cudaError_t launch_backward_ext_mw_q(const DevTopo& T, const DevPtrs& D, int t, cudaStream_t s) {
  size_t smem = SM_BYTES(T);
  cudaError_t e = cudaFuncSetAttribute(k_backward_ext_mw<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_backward_ext_mw<Q><<<T.Bp / 32, 128, smem, s>>>(T, D, t);
  return cudaGetLastError();
}
cudaError_t launch_backward_ext(const DevTopo& T, const DevPtrs& D, int t, cudaStream_t s) {
  if (T.topo_id == QuadrupedTopo::id && D.tape_full && !T.one_warp && !getenv("DP_SINGLE_WARP_BACKWARD"))
    return launch_backward_ext_mw_q<QuadrupedTopo>(T, D, t, s);
  if (T.topo_id == QuadrupedTopo::id) return launch_backward_ext_q<QuadrupedTopo>(T, D, t, s);
  return launch_backward_ext_q<DynTopo>(T, D, t, s);
}
