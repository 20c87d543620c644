// Internal layout of a dp_world (shared by the C-ABI translation units of libdphys).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/dp.h"
#include "dp_device.cuh"

// bf16 layouts of a wide controller (offsets in elements): W1 [h1][k0p], W2 [h2][h1], W3 [8][h2]
// and the transposes W3t [h2][16], W2t [h1][h2], W1t [k0p][h1].
struct ExtLayout {
  int k0p, h1, h2, no;
  size_t w1, w2, w3, w3t, w2t, w1t, size;
};

struct dp_world {
  DevTopo Tf, Tb;  // same topology; forward / backward shared-memory layouts
  DevPtrs D;
  cudaStream_t stream = nullptr;
  int device = 0;  // the CUDA device current at creation (the world's buffers live there)
  int B = 0, Bp = 0, nf = 0;
  int64_t n_params = 0;
  int w_total = 0;
  float* x0 = nullptr;
  float* Wmaster = nullptr;
  float *Wt = nullptr, *Wn = nullptr, *Wb = nullptr;
  __nv_bfloat16* Wtc = nullptr;  // tensor-core layouts of the controller (DevTopo.mlp_tc)
  bool ws_capable = false;       // created with room for the warm start (tape lam0 record)
  float* ws_master = nullptr;    // warm-start parameters [DP_WS_PARAMS]
  __nv_bfloat16* ws_tc = nullptr;
  float* ws_b = nullptr;
  unsigned long long* harvest_count = nullptr;
  float* resid = nullptr;        // per-instance residual sums [Bp]
  float ws_alpha = 0.7f;
  bool resid_on = false;
  // wide controller (DevTopo.ext_ctrl)
  ExtLayout ext{};
  __nv_bfloat16 *ext_w = nullptr, *ext_h1 = nullptr, *ext_h2 = nullptr;
  float *ext_d1 = nullptr, *ext_d2 = nullptr;
  int resid_steps = 0;
  float* stage = nullptr;      // device staging buffer for user-layout inputs/outputs
  size_t stage_floats = 0;
  float* dW_stage = nullptr;   // [n_params]
  float* partial = nullptr;    // dW split partials
  size_t partial_floats = 0;
  int splits = 1;
  std::vector<void*> allocs;
  int t_now = 0;
  bool have_rollout = false;
  int32_t kind[DPK_MAXSLOT], colour[DPK_MAXSLOT];
};

// Records `msg` as the thread's last error and returns `s`.
dp_status dp_internal_fail(dp_status s, const char* msg);

// Wide-controller path (dp_ext.cu).
cudaError_t launch_prep_ext(const ExtLayout& Lo, int K0, const float* W, __nv_bfloat16* out, cudaStream_t s);
cudaError_t ext_forward(dp_world* w, const DevTopo& T, const DevPtrs& D, int t0, int nsteps, int rollout, int record);
cudaError_t ext_backward(dp_world* w, const DevTopo& T, const DevPtrs& D);
cudaError_t tc_weight_grad(dp_world* w, const DevTopo& T, const DevPtrs& D, float* dst);
