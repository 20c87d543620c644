// dp_backward_noalloc: the reverse pass of dp_backward for callers that must not allocate
// device memory while they run. The split-K partial sums of the controller-gradient reduction
// live in a fixed static device array instead of a buffer owned by the world.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/dp.h"
#include "dp_kernels.h"
#include "dp_world.h"

// One array per GPU that loads the library, held until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[DP_NOALLOC_SCRATCH_FLOATS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the static array on the world's device, which must be current. In host
// code the array's name is only a host-side stand-in, so the address is looked up once per
// device with that device current, and reused afterwards (a cudaDeviceReset after that first
// call would reload the module and may move the array: not supported).
dp_status scratch_address(int world_dev, float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dp_internal_fail(DP_ECUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
  if (dev != world_dev)
    return dp_internal_fail(DP_EINVAL, ("the world's device " + std::to_string(world_dev) + " is not current (device " +
                                        std::to_string(dev) + " is)").c_str());
  if (dev < 0 || dev >= kMaxDevices) return dp_internal_fail(DP_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return dp_internal_fail(DP_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return DP_OK;
}

#define CUN(call)                                                                                              \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) return dp_internal_fail(DP_ECUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)

}  // namespace

extern "C" dp_status dp_backward_noalloc(dp_world* w, const float* dloss, float* dW) {
  if (!w) return dp_internal_fail(DP_EINVAL, "world is NULL");
  if (!w->have_rollout) return dp_internal_fail(DP_ESTATE, "dp_backward_noalloc needs a preceding dp_rollout");
  if (w->Tb.ext_ctrl) return dp_internal_fail(DP_EINVAL, "dp_backward_noalloc does not serve wide controllers; use dp_backward");
  if (!dloss || !dW) return dp_internal_fail(DP_EINVAL, "dloss and dW are required");
  if (w->n_params == 0) return dp_internal_fail(DP_EINVAL, "the world has no controller");
  const DevTopo& T = w->Tb;
  const int nl = T.n_layers + (T.skip ? 1 : 0);
  // every layer must fit the static array with at least one split; checked before any launch
  for (int l = 0; l < nl; ++l) {
    const bool sk = l == T.n_layers;
    const size_t mc = (size_t)(sk ? T.widths[0] : T.widths[l]) * (size_t)(sk ? T.widths[T.n_layers] : T.widths[l + 1]);
    if (mc > (size_t)DP_NOALLOC_SCRATCH_FLOATS)
      return dp_internal_fail(DP_EINVAL, ("controller layer with " + std::to_string(mc) +
                                          " weights exceeds the static scratch of " +
                                          std::to_string(DP_NOALLOC_SCRATCH_FLOATS) + " floats").c_str());
  }
  float* scratch = nullptr;
  dp_status st = scratch_address(w->device, &scratch);
  if (st != DP_OK) return st;
  DevPtrs& D = w->D;
  CUN(cudaMemcpyAsync(w->stage, dloss, sizeof(float) * w->B, cudaMemcpyDefault, w->stream));
  CUN(launch_pad_scalar(w->B, w->Bp, w->stage, D.dloss, w->stream));
  CUN(cudaMemsetAsync(D.grad_prm, 0, sizeof(float) * (size_t)T.n_pfields * w->Bp, w->stream));
  CUN(launch_backward(T, D, w->stream));
  const size_t N = (size_t)T.horizon * w->Bp;
  size_t off = 0;
  for (int l = 0; l < nl; ++l) {
    const bool sk = l == T.n_layers;
    const int ni = sk ? T.widths[0] : T.widths[l];
    const int no_ = sk ? T.widths[T.n_layers] : T.widths[l + 1];
    const size_t mc = (size_t)no_ * ni;
    // Every partial a reduction reads is written earlier in the same call, so the contents left
    // by a previous call never leak into this one.
    const int splits = (int)std::max<size_t>(1, std::min<size_t>((size_t)w->splits, DP_NOALLOC_SCRATCH_FLOATS / mc));
    const size_t chunk = ((N + splits - 1) / splits + 15) / 16 * 16;
    const float* del = D.dump + (size_t)T.dump_del[sk ? T.n_layers - 1 : l] * N;
    const float* act = D.dump + (size_t)T.dump_act[sk ? 0 : l] * N;
    CUN(launch_dw(del, act, no_, ni, N, scratch, splits, chunk, w->stream));
    CUN(launch_sum_splits(scratch, splits, mc, w->dW_stage + off, w->stream));
    off += mc;
    CUN(launch_rowsum(del, no_, N, scratch, splits, chunk, w->stream));
    CUN(launch_sum_splits(scratch, splits, (size_t)no_, w->dW_stage + off, w->stream));
    off += no_;
  }
  CUN(cudaMemcpyAsync(dW, w->dW_stage, sizeof(float) * w->n_params, cudaMemcpyDefault, w->stream));
  return DP_OK;
}
