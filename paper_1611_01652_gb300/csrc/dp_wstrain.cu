// Learned warm start: training and stand-alone inference of the 16-64-64-3 network on the GPU.
// The network maps the 16 features of a contact to its (normal, t1, t2) impulses; it is trained
// on rows harvested from cold-start rollouts (features, converged impulses) by minimising the
// mean squared error. Forward and reverse passes run on the bfloat16 tensor cores with the
// storage points of the in-step inference (inputs, weights and hidden activations in bfloat16,
// fp32 accumulation, straight-through rounding in reverse mode); the weight gradient is the
// split-K reduction of the stored deltas against the stored activations; Adam updates the fp32
// master weights.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dp.h"
#include "dp_kernels.h"
#include "dp_mma.cuh"
#include "dp_world.h"

namespace {

constexpr int WS_ROW = 19;       // harvested row: 16 features, 3 impulses
constexpr int WS_WARPS = 4;      // warps per block of the row kernels
constexpr int ACT_ROWS = WsTC::K0 + WsTC::H1 + WsTC::H2;   // stored activations per row
constexpr int DEL_ROWS = WsTC::H1 + WsTC::H2 + WsTC::NO;   // stored deltas per row

// Flat fp32 parameters -> tensor-core layouts (zero padded) and the bias array.
__global__ void k_ws_prep(const float* __restrict__ W, __nv_bfloat16* tc, float* bias) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < WsTC::BSIZE) {
    float v = 0.f;
    if (p < WsTC::B2) v = W[WsTC::F_B1 + p];
    else if (p < WsTC::B3) v = W[WsTC::F_B2 + p - WsTC::B2];
    else if (p - WsTC::B3 < WsTC::NO) v = W[WsTC::F_B3 + p - WsTC::B3];
    bias[p] = v;
  }
  if (p >= WsTC::SIZE) return;
  auto w1 = [&](int o, int i) { return W[WsTC::F_W1 + o * WsTC::K0 + i]; };
  auto w2 = [&](int o, int i) { return W[WsTC::F_W2 + o * WsTC::H1 + i]; };
  auto w3 = [&](int o, int i) { return o < WsTC::NO ? W[WsTC::F_W3 + o * WsTC::H2 + i] : 0.f; };
  float v;
  if (p < WsTC::W2) {  // W1 [64][16]
    v = w1(p / 16, p % 16);
  } else if (p < WsTC::W3) {  // W2 [64][64]
    const int q = p - WsTC::W2;
    v = w2(q / WsTC::H1, q % WsTC::H1);
  } else if (p < WsTC::W3T) {  // W3 [8][64]
    const int q = p - WsTC::W3;
    v = w3(q / WsTC::H2, q % WsTC::H2);
  } else if (p < WsTC::W2T) {  // W3^T [64][16]
    const int q = p - WsTC::W3T;
    v = w3(q % 16, q / 16);
  } else if (p < WsTC::W1T) {  // W2^T [64][64]
    const int q = p - WsTC::W2T;
    v = w2(q % WsTC::H2, q / WsTC::H2);
  } else {  // W1^T [16][64]
    const int q = p - WsTC::W1T;
    v = w1(q % WsTC::H1, q / WsTC::H1);
  }
  tc[p] = __float2bfloat16_rn(v);
}

// Inference: y[n][3] for features x[n][stride] (first 16 columns).
__global__ void __launch_bounds__(32 * WS_WARPS) k_ws_infer(const __nv_bfloat16* __restrict__ tc,
                                                             const float* __restrict__ bias,
                                                             const float* __restrict__ x, int stride, long long n,
                                                             float* __restrict__ y) {
  const long long base = ((long long)blockIdx.x * WS_WARPS + (threadIdx.x >> 5)) * 32;
  if (base >= n) return;  // whole warp leaves together
  mlp3_forward<WsTC::K0, WsTC::H1, WsTC::H2, WsTC::NO>(
      WsTC::K0, WsTC::NO,
      [&](int f, int r) { return base + r < n ? x[(base + r) * stride + f] : 0.f; }, tc + WsTC::W1, bias + WsTC::B1,
      tc + WsTC::W2, bias + WsTC::B2, tc + WsTC::W3, bias + WsTC::B3,
      [&](int f, int r, float v) {
        if (base + r < n) y[(base + r) * WsTC::NO + f] = v;
      },
      [](int, int, int, float) {});
}

// Forward and reverse pass of the squared-error loss on 32 rows per warp. Stores, per row
// column (stride np = n rounded up to 32): act = [bf16 features (16), hidden 1 (64), hidden 2
// (64)], del = [delta hidden 1 (64), delta hidden 2 (64), delta output (3)], and the warp's
// partial sum of squared errors. Padded rows have zero deltas.
__global__ void __launch_bounds__(32 * WS_WARPS) k_ws_fwdbwd(const __nv_bfloat16* __restrict__ tc,
                                                              const float* __restrict__ bias,
                                                              const float* __restrict__ rows, long long n,
                                                              long long np, float inv_n, float* __restrict__ act,
                                                              float* __restrict__ del, float* __restrict__ loss_part) {
  __shared__ float ys[WS_WARPS][WsTC::NO][32];
  __shared__ float ubs[WS_WARPS][WsTC::NO][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * WS_WARPS + warp;
  const long long base = wid * 32;
  if (base >= np) return;
  const long long me = base + lane;
  const bool valid = me < n;
  for (int f = 0; f < WsTC::K0; ++f) act[(size_t)f * np + me] = valid ? bf16r(rows[me * WS_ROW + f]) : 0.f;
  auto col = [&](int r) { return base + r; };
  mlp3_forward<WsTC::K0, WsTC::H1, WsTC::H2, WsTC::NO>(
      WsTC::K0, WsTC::NO,
      [&](int f, int r) { return col(r) < n ? rows[col(r) * WS_ROW + f] : 0.f; }, tc + WsTC::W1, bias + WsTC::B1,
      tc + WsTC::W2, bias + WsTC::B2, tc + WsTC::W3, bias + WsTC::B3,
      [&](int f, int r, float v) { ys[warp][f][r] = v; },
      [&](int l, int f, int r, float v) {
        act[(size_t)((l == 1 ? WsTC::K0 : WsTC::K0 + WsTC::H1) + f) * np + col(r)] = col(r) < n ? v : 0.f;
      });
  __syncwarp();
  float e = 0.f;
  for (int k = 0; k < WsTC::NO; ++k) {
    const float d = valid ? ys[warp][k][lane] - rows[me * WS_ROW + WsTC::K0 + k] : 0.f;
    e += d * d;
    const float g = 2.f * d * inv_n;
    ubs[warp][k][lane] = g;
    del[(size_t)(WsTC::H1 + WsTC::H2 + k) * np + me] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0) loss_part[wid] = e;
  __syncwarp();
  mlp3_backward<WsTC::K0, WsTC::H1, WsTC::H2, WsTC::NO>(
      WsTC::K0, WsTC::NO,
      [&](int f, int r) { return ubs[warp][f][r]; }, tc + WsTC::W3T, tc + WsTC::W2T, tc + WsTC::W1T,
      [&](int l, int f, int r) {
        return act[(size_t)((l == 1 ? WsTC::K0 : WsTC::K0 + WsTC::H1) + f) * np + col(r)] > 0.f;
      },
      [&](int l, int f, int r, float v) { del[(size_t)((l == 1 ? 0 : WsTC::H1) + f) * np + col(r)] = v; },
      [](int, int, float) {});
}

// Deterministic sum of count values by one block (fixed strided order, then a tree).
__global__ void k_sum_block(const float* __restrict__ x, long long count, float scale, float* out) {
  __shared__ float red[256];
  float s = 0.f;
  for (long long k = threadIdx.x; k < count; k += blockDim.x) s += x[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// Adam (Kingma and Ba, 2015) on fp32 parameters with bias-corrected moments.
__global__ void k_adam(float* W, const float* __restrict__ g, float* m, float* v, long long count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  W[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

long long round32(long long n) { return (n + 31) / 32 * 32; }
int splits_for(long long np) { return (int)std::min<long long>(256, (np + 16383) / 16384); }

// Workspace carve-up (floats): tensor-core weights, biases, activations, deltas, split-K
// partials, per-warp loss partials.
struct WsWork {
  __nv_bfloat16* tc;
  float *bias, *act, *del, *partial, *loss_part;
};
WsWork carve(float* work, long long n) {
  const long long np = round32(n);
  WsWork w;
  float* p = work;
  w.tc = reinterpret_cast<__nv_bfloat16*>(p);
  p += (WsTC::SIZE + 1) / 2 + 64;
  w.bias = p;
  p += WsTC::BSIZE + 56;
  w.act = p;
  p += (size_t)ACT_ROWS * np;
  w.del = p;
  p += (size_t)DEL_ROWS * np;
  w.partial = p;
  p += (size_t)splits_for(np) * WsTC::H1 * WsTC::H2;
  w.loss_part = p;
  return w;
}

}  // namespace

cudaError_t launch_ws_prep(const float* W, __nv_bfloat16* tc, float* bias, cudaStream_t s) {
  k_ws_prep<<<(WsTC::SIZE + 255) / 256, 256, 0, s>>>(W, tc, bias);
  return cudaGetLastError();
}

extern "C" {

int64_t dp_ws_workspace_floats(int64_t n) {
  if (n < 0) return -1;
  const long long np = round32(std::max<long long>(n, 1));
  return (WsTC::SIZE + 1) / 2 + 64 + WsTC::BSIZE + 56 + (long long)(ACT_ROWS + DEL_ROWS) * np +
         (long long)splits_for(np) * WsTC::H1 * WsTC::H2 + np / 32 + 32;
}

int32_t dp_ws_param_count(void) { return WsTC::PARAMS; }

dp_status dp_ws_forward(const float* W, const float* feats, int64_t n, float* y, float* work, void* stream) {
  if (!W || !feats || !y || !work || n < 0) return dp_internal_fail(DP_EINVAL, "dp_ws_forward: NULL pointer or n < 0");
  if (n == 0) return DP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  WsWork w = carve(work, n);
  k_ws_prep<<<(WsTC::SIZE + 255) / 256, 256, 0, s>>>(W, w.tc, w.bias);
  const long long warps = round32(n) / 32;
  k_ws_infer<<<(unsigned)((warps + WS_WARPS - 1) / WS_WARPS), 32 * WS_WARPS, 0, s>>>(w.tc, w.bias, feats, WsTC::K0, n, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DP_OK : dp_internal_fail(DP_ECUDA, cudaGetErrorString(e));
}

dp_status dp_ws_loss_grad(const float* W, const float* rows, int64_t n, float* loss, float* dW, float* work,
                          void* stream) {
  if (!W || !rows || !loss || !dW || !work || n <= 0)
    return dp_internal_fail(DP_EINVAL, "dp_ws_loss_grad: NULL pointer or n <= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const long long np = round32(n);
  WsWork w = carve(work, n);
  k_ws_prep<<<(WsTC::SIZE + 255) / 256, 256, 0, s>>>(W, w.tc, w.bias);
  const long long warps = np / 32;
  k_ws_fwdbwd<<<(unsigned)((warps + WS_WARPS - 1) / WS_WARPS), 32 * WS_WARPS, 0, s>>>(
      w.tc, w.bias, rows, n, np, 1.f / (float)n, w.act, w.del, w.loss_part);
  k_sum_block<<<1, 256, 0, s>>>(w.loss_part, warps, 1.f / (float)n, loss);
  // dW_l = sum over rows of delta_l (x) act_l, db_l = sum of delta_l
  const int splits = splits_for(np);
  const size_t chunk = (size_t)((np + splits - 1) / splits + 15) / 16 * 16;
  struct L { int M, C, act_row, del_row, fw, fb; };
  const L layers[3] = {{WsTC::H1, WsTC::K0, 0, 0, WsTC::F_W1, WsTC::F_B1},
                       {WsTC::H2, WsTC::H1, WsTC::K0, WsTC::H1, WsTC::F_W2, WsTC::F_B2},
                       {WsTC::NO, WsTC::H2, WsTC::K0 + WsTC::H1, WsTC::H1 + WsTC::H2, WsTC::F_W3, WsTC::F_B3}};
  for (const L& l : layers) {
    const float* dl = w.del + (size_t)l.del_row * np;
    const float* al = w.act + (size_t)l.act_row * np;
    cudaError_t e = launch_dw(dl, al, l.M, l.C, (size_t)np, w.partial, splits, chunk, s);
    if (e == cudaSuccess) e = launch_sum_splits(w.partial, splits, (size_t)l.M * l.C, dW + l.fw, s);
    if (e == cudaSuccess) e = launch_rowsum(dl, l.M, (size_t)np, w.partial, splits, chunk, s);
    if (e == cudaSuccess) e = launch_sum_splits(w.partial, splits, (size_t)l.M, dW + l.fb, s);
    if (e != cudaSuccess) return dp_internal_fail(DP_ECUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DP_OK : dp_internal_fail(DP_ECUDA, cudaGetErrorString(e));
}

dp_status dp_ws_adam(float* W, const float* dW, float* m, float* v, int64_t count, int32_t step, float lr, float beta1,
                     float beta2, float eps, void* stream) {
  if (!W || !dW || !m || !v || count < 0 || step < 1)
    return dp_internal_fail(DP_EINVAL, "dp_ws_adam: NULL pointer, count < 0 or step < 1");
  if (count == 0) return DP_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(W, dW, m, v, count, lr, beta1, beta2, eps,
                                                                            c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DP_OK : dp_internal_fail(DP_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
