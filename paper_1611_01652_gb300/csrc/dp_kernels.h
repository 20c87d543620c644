// Host-side launchers of the kernels in dp_kernels.cu, dp_fwd.cu, dp_fwd_mw.cu, dp_bwd.cu,
// dp_bwd_mw.cu and dp_bwd_ext.cu (internal to libdphys).
#pragma once
#include <cuda_runtime.h>

#include "dp_device.cuh"

cudaError_t launch_prep_weights(const DevTopo& T, const float* W, float* Wt, float* Wn, float* bias, cudaStream_t s);
cudaError_t launch_prep_weights_tc(const DevTopo& T, const float* W, __nv_bfloat16* Wc, cudaStream_t s);
cudaError_t launch_ws_prep(const float* W, __nv_bfloat16* tc, float* bias, cudaStream_t s);
cudaError_t launch_scale_out(int B, const float* src, float scale, float* dst, cudaStream_t s);
cudaError_t launch_state_in(int B, int Bp, int nf, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_state_out(int B, int Bp, int nf, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_param_out(int B, int Bp, int o, int n, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_param_in(int B, int Bp, int o, int n, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_pad_scalar(int B, int Bp, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_forward(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps, int rollout,
                           int record, cudaStream_t s);
cudaError_t launch_forward_mw_quadruped(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps,
                                        int rollout, cudaStream_t s);
cudaError_t launch_forward_mw_arm(const DevTopo& T, const DevPtrs& D, const float* x0, int t0, int nsteps,
                                  int rollout, cudaStream_t s);
cudaError_t launch_backward(const DevTopo& T, const DevPtrs& D, cudaStream_t s);
cudaError_t launch_backward_mw_quadruped(const DevTopo& T, const DevPtrs& D, cudaStream_t s);
cudaError_t launch_backward_mw_arm(const DevTopo& T, const DevPtrs& D, cudaStream_t s);
cudaError_t launch_backward_ext(const DevTopo& T, const DevPtrs& D, int t, cudaStream_t s);
cudaError_t launch_dw(const float* del, const float* act, int M, int C, size_t N, float* partial, int splits,
                      size_t chunk, cudaStream_t s);
cudaError_t launch_rowsum(const float* del, int M, size_t N, float* partial, int splits, size_t chunk, cudaStream_t s);
cudaError_t launch_check_grads(int B, int Bp, int nf, int np, const float* gs, const float* gp, int* status,
                               cudaStream_t s);
cudaError_t launch_sum_splits(const float* partial, int splits, size_t count, float* out, cudaStream_t s);
int match_compiled_topology(const DevTopo& T, int nb, int nj, int ns, int np, const int* jtype, const int* jbody,
                            const int* jflags, const int* sbody, const int* pair);
// hidden width of the tensor-core controller the compiled topology's kernels carry (0: none)
int compiled_ctrl_width(int topo_id);
