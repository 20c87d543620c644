// Wide controllers (e.g. 64-1024-1024-8, 1.1 M parameters): the dense network of Eq. g is too wide
// to live on chip beside a warp's 32 robots, so it runs between step launches as batched products
// over all instances on the bfloat16 tensor cores (mma.sync m16n8k16, fp32 accumulation). A warp
// computes a 32-row x (8 NT)-column tile of C = A B^T, A row-major [M][K] (bf16, or fp32 deltas
// split into bf16 hi + lo), B row-major [N][K] bf16; the epilogue applies the layer's bias, ReLU
// and bfloat16 storage, the ReLU mask of the reverse pass, and writes the activation/delta dump
// (feature-major) that the weight-gradient reduction reads.
//
// Forward, step t: s_t (bf16, written by the previous step launch) -> h1 -> h2 -> u_t, then the
// step launch reads u_t and writes s_{t+1}. Reverse, step t: the step launch reverses step t down
// to the adjoint of u_t, then delta_2 = (u_bar W3) . [h2 > 0], delta_1 = (delta_2 W2) . [h1 > 0],
// s_bar = delta_1 W1, read by the next (earlier) step launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dp_kernels.h"
#include "dp_mma.cuh"
#include "dp_world.h"

namespace {

enum { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_BWD_HIDDEN = 2, EPI_BWD_IN = 3 };

struct GemmEpi {
  int kind;
  const float* bias;      // [N] (forward)
  int nvalid;             // real columns (forward output)
  void* out;              // bf16 (EPI_FWD_HIDDEN) or fp32, row-major with leading dimension ldo
  int ldo;
  float* dump;            // feature-major dump [row][ncol], column col0 + m; or nullptr
  int dump_row;
  size_t ncol, col0;
  const float* mask;      // EPI_BWD_HIDDEN: dump rows of the layer's input activations
  int mask_row;
};

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int NT, bool AF32>
__global__ void __launch_bounds__(128) k_ctrl_gemm(const void* __restrict__ Av, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int M, int N, int K,
                                                   const GemmEpi e) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int mw = M / 32, nw = N / (8 * NT);
  if (warp >= mw * nw) return;  // whole warp
  const int m0 = (warp % mw) * 32, n0 = (warp / mw) * (8 * NT);
  float acc[2][NT][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int kt = 0; kt < K / 16; ++kt) {
    const int c = kt * 16 + 2 * q;
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = m0 + mt * 16 + g, r1 = r0 + 8;
      if constexpr (AF32) {
        const float* A = static_cast<const float*>(Av);
        const float2 x[4] = {__ldg(reinterpret_cast<const float2*>(A + (size_t)r0 * lda + c)),
                             __ldg(reinterpret_cast<const float2*>(A + (size_t)r1 * lda + c)),
                             __ldg(reinterpret_cast<const float2*>(A + (size_t)r0 * lda + c + 8)),
                             __ldg(reinterpret_cast<const float2*>(A + (size_t)r1 * lda + c + 8))};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float hx = bf16_round(x[j].x), hy = bf16_round(x[j].y);
          ah[mt][j] = pack_bf16(hx, hy);
          al[mt][j] = pack_bf16(x[j].x - hx, x[j].y - hy);
        }
      } else {
        const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(Av);
        ah[mt][0] = __ldg(reinterpret_cast<const unsigned int*>(A + (size_t)r0 * lda + c));
        ah[mt][1] = __ldg(reinterpret_cast<const unsigned int*>(A + (size_t)r1 * lda + c));
        ah[mt][2] = __ldg(reinterpret_cast<const unsigned int*>(A + (size_t)r0 * lda + c + 8));
        ah[mt][3] = __ldg(reinterpret_cast<const unsigned int*>(A + (size_t)r1 * lda + c + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      load_b(B, K, n0 + nt * 8, kt * 16, b0, b1);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        mma_bf16_16816(acc[mt][nt], ah[mt], b0, b1);
        if constexpr (AF32) mma_bf16_16816(acc[mt][nt], al[mt], b0, b1);
      }
    }
  }
  // epilogue: element (m, n) of fragment position k: rows g / g+8, columns 2q / 2q+1
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int m = m0 + mt * 16 + g + (k >= 2 ? 8 : 0);
        const int n = n0 + nt * 8 + 2 * q + (k & 1);
        float v = acc[mt][nt][k];
        if (e.kind == EPI_FWD_HIDDEN) {
          v = bf16_round(fmaxf(v + e.bias[n], 0.f));
          static_cast<__nv_bfloat16*>(e.out)[(size_t)m * e.ldo + n] = __float2bfloat16_rn(v);
        } else if (e.kind == EPI_FWD_OUT) {
          v = n < e.nvalid ? v + e.bias[n] : 0.f;
          static_cast<float*>(e.out)[(size_t)m * e.ldo + n] = v;
        } else if (e.kind == EPI_BWD_HIDDEN) {
          if (!(e.mask[(size_t)(e.mask_row + n) * e.ncol + e.col0 + m] > 0.f)) v = 0.f;
          static_cast<float*>(e.out)[(size_t)m * e.ldo + n] = v;
        } else {
          static_cast<float*>(e.out)[(size_t)m * e.ldo + n] = v;
        }
        if (e.dump && n < e.nvalid) e.dump[(size_t)(e.dump_row + n) * e.ncol + e.col0 + m] = v;
      }
}

template <int NT, bool AF32>
cudaError_t gemm(const void* A, int lda, const __nv_bfloat16* B, int M, int N, int K, const GemmEpi& e, cudaStream_t s) {
  const long long warps = (long long)(M / 32) * (N / (8 * NT));
  k_ctrl_gemm<NT, AF32><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(A, lda, B, M, N, K, e);
  return cudaGetLastError();
}

// Flat fp32 master weights (per layer W[out][in] then b[out]) -> bf16 layouts of the three
// layers and of their transposes, zero padded (ExtLayout).
__global__ void k_prep_ext(const ExtLayout Lo, int K0, const float* __restrict__ W, __nv_bfloat16* __restrict__ out) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lo.size) return;
  const int H1 = Lo.h1, H2 = Lo.h2, NO = Lo.no, K0p = Lo.k0p;
  const size_t m1 = (size_t)K0 * H1 + H1, m2 = m1 + (size_t)H1 * H2 + H2;
  auto w1 = [&](int o, int i) { return i < K0 ? W[(size_t)o * K0 + i] : 0.f; };
  auto w2 = [&](int o, int i) { return W[m1 + (size_t)o * H1 + i]; };
  auto w3 = [&](int o, int i) { return o < NO ? W[m2 + (size_t)o * H2 + i] : 0.f; };
  float v;
  if (p < Lo.w2) {
    const size_t q = p - Lo.w1;
    v = w1((int)(q / K0p), (int)(q % K0p));
  } else if (p < Lo.w3) {
    const size_t q = p - Lo.w2;
    v = w2((int)(q / H1), (int)(q % H1));
  } else if (p < Lo.w3t) {
    const size_t q = p - Lo.w3;
    v = w3((int)(q / H2), (int)(q % H2));
  } else if (p < Lo.w2t) {
    const size_t q = p - Lo.w3t;
    v = w3((int)(q % 16), (int)(q / 16));
  } else if (p < Lo.w1t) {
    const size_t q = p - Lo.w2t;
    v = w2((int)(q % H2), (int)(q / H2));
  } else {
    const size_t q = p - Lo.w1t;
    v = w1((int)(q % H1), (int)(q / H1));
  }
  out[p] = __float2bfloat16_rn(v);
}

}  // namespace

cudaError_t launch_prep_ext(const ExtLayout& Lo, int K0, const float* W, __nv_bfloat16* out, cudaStream_t s) {
  k_prep_ext<<<(unsigned)((Lo.size + 255) / 256), 256, 0, s>>>(Lo, K0, W, out);
  return cudaGetLastError();
}

// Controller products of step t (forward): s_t -> h1 -> h2 -> u_t; with `record` the activations
// also go to the dump columns of step t.
cudaError_t ext_forward_products(dp_world* w, const DevTopo& T, const DevPtrs& D, int t, bool record) {
  const ExtLayout& Lo = w->ext;
  const int M = T.Bp;
  const size_t ncol = (size_t)T.horizon * T.Bp, col0 = (size_t)t * T.Bp;
  const int slot = t % T.horizon;
  GemmEpi e{};
  e.ncol = ncol;
  e.col0 = col0;
  e.kind = EPI_FWD_HIDDEN;
  e.bias = D.bias + T.w_off[0];
  e.nvalid = Lo.h1;
  e.out = w->ext_h1;
  e.ldo = Lo.h1;
  e.dump = record ? D.dump : nullptr;
  e.dump_row = T.dump_act[1];
  cudaError_t r = gemm<8, false>(D.s_ext, Lo.k0p, w->ext_w + Lo.w1, M, Lo.h1, Lo.k0p, e, w->stream);
  if (r != cudaSuccess) return r;
  e.bias = D.bias + T.w_off[1];
  e.nvalid = Lo.h2;
  e.out = w->ext_h2;
  e.ldo = Lo.h2;
  e.dump_row = T.dump_act[2];
  r = gemm<8, false>(w->ext_h1, Lo.h1, w->ext_w + Lo.w2, M, Lo.h2, Lo.h1, e, w->stream);
  if (r != cudaSuccess) return r;
  e.kind = EPI_FWD_OUT;
  e.bias = D.bias + T.w_off[2];
  e.nvalid = Lo.no;
  e.out = D.u_ext + (size_t)slot * M * T.ext_nop;
  e.ldo = T.ext_nop;
  e.dump_row = T.dump_act[3];
  return gemm<1, false>(w->ext_h2, Lo.h2, w->ext_w + Lo.w3, M, 8, Lo.h2, e, w->stream);
}

// Controller products of step t (reverse): u_bar -> delta_2 -> delta_1 -> s_bar, deltas to the dump.
cudaError_t ext_backward_products(dp_world* w, const DevTopo& T, const DevPtrs& D, int t) {
  const ExtLayout& Lo = w->ext;
  const int M = T.Bp;
  GemmEpi e{};
  e.ncol = (size_t)T.horizon * T.Bp;
  e.col0 = (size_t)t * T.Bp;
  e.kind = EPI_BWD_HIDDEN;
  e.nvalid = Lo.h2;
  e.out = w->ext_d2;
  e.ldo = Lo.h2;
  e.dump = D.dump;
  e.dump_row = T.dump_del[1];
  e.mask = D.dump;
  e.mask_row = T.dump_act[2];
  cudaError_t r = gemm<8, true>(D.ub_ext, 16, w->ext_w + Lo.w3t, M, Lo.h2, 16, e, w->stream);
  if (r != cudaSuccess) return r;
  e.nvalid = Lo.h1;
  e.out = w->ext_d1;
  e.ldo = Lo.h1;
  e.dump_row = T.dump_del[0];
  e.mask_row = T.dump_act[1];
  r = gemm<8, true>(w->ext_d2, Lo.h2, w->ext_w + Lo.w2t, M, Lo.h1, Lo.h2, e, w->stream);
  if (r != cudaSuccess) return r;
  e.kind = EPI_BWD_IN;
  e.nvalid = Lo.k0p;
  e.out = const_cast<float*>(D.sbar_ext);
  e.ldo = Lo.k0p;
  e.dump = nullptr;
  return gemm<8, true>(w->ext_d1, Lo.h1, w->ext_w + Lo.w1t, M, Lo.k0p, Lo.h1, e, w->stream);
}

// A rollout part with the wide controller: the features of the start state, then per step the
// controller products and one step launch. rollout: 1 = a whole recorded rollout from x0, 0 =
// dp_step from the current state.
cudaError_t ext_forward(dp_world* w, const DevTopo& T, const DevPtrs& D, int t0, int nsteps, int rollout, int record) {
  const int mode = rollout ? 2 : 0;
  cudaError_t r = launch_forward(T, D, w->x0, t0, 0, mode, record, w->stream);  // features of the start state
  for (int k = 0; k < nsteps && r == cudaSuccess; ++k) {
    const int t = t0 + k;
    r = ext_forward_products(w, T, D, t, record != 0);
    if (r == cudaSuccess) r = launch_forward(T, D, w->x0, t, 1, mode, record, w->stream);
  }
  return r;
}

// Reverse mode with the wide controller, last step first; the state adjoint accumulates in
// grad_state0.
cudaError_t ext_backward(dp_world* w, const DevTopo& T, const DevPtrs& D) {
  cudaError_t r = cudaMemsetAsync(D.grad_state0, 0, sizeof(float) * (size_t)18 * T.nb * T.Bp, w->stream);
  for (int t = T.horizon - 1; t >= -1 && r == cudaSuccess; --t) {
    r = launch_backward_ext(T, D, t, w->stream);
    if (r == cudaSuccess && t >= 0) r = ext_backward_products(w, T, D, t);
  }
  return r;
}
