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
#include <cmath>
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
  void* out;              // bf16 (EPI_FWD_HIDDEN; EPI_BWD_HIDDEN: high plane) or fp32, row-major, leading dim ldo
  __nv_bfloat16* out_lo;  // EPI_BWD_HIDDEN: low plane (value minus its bfloat16 rounding)
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
          const float hi = bf16_round(v);
          static_cast<__nv_bfloat16*>(e.out)[(size_t)m * e.ldo + n] = __float2bfloat16_rn(hi);
          e.out_lo[(size_t)m * e.ldo + n] = __float2bfloat16_rn(v - hi);
        } else {
          static_cast<float*>(e.out)[(size_t)m * e.ldo + n] = v;
        }
        if (e.dump && n < e.nvalid) e.dump[(size_t)(e.dump_row + n) * e.ncol + e.col0 + m] = v;
      }
}

// ---------------------------------------------------------------------------------------------
// Tiled products: a CTA of 8 warps computes a 128 x BN tile of C = A B^T; A (bf16, optionally a
// second bf16 plane holding the low part of a split fp32 operand) and B are staged through
// shared memory in 32-column k-chunks by cp.async (double buffered, rows past M zero-filled),
// fragments are read with ldmatrix from rows padded to 40 halves (80 bytes: the 8 row addresses
// of an 8x8 matrix fall in 8 different 16-byte bank groups).
constexpr int TBM = 128, TBK = 32, TLDS = 40;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void ldsm_x4(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}


template <int BN, bool SPLIT>
__global__ void __launch_bounds__(256) k_tc_gemm(const __nv_bfloat16* __restrict__ Ahi, const __nv_bfloat16* __restrict__ Alo,
                                                 const __nv_bfloat16* __restrict__ B, int M, int N, int K, const GemmEpi e) {
  constexpr int WN = BN / 32, WM = 8 / WN, WTM = TBM / WM, MT = WTM / 16;
  constexpr int APL = TBM * TLDS, BPL = BN * TLDS;  // halves per plane and stage
  extern __shared__ __align__(16) unsigned char tc_smem[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(tc_smem);       // [2][SPLIT+1][APL]
  __nv_bfloat16* sB = sA + 2 * (SPLIT ? 2 : 1) * APL;                    // [2][BPL]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
  const int wr = (warp / WN) * WTM, wc = (warp % WN) * 32;
  auto load = [&](int kc, int buf) {
    const int k0 = kc * TBK;
    for (int c = tid; c < TBM * 4; c += 256) {
      const int r = c >> 2, col = (c & 3) * 8;
      const bool ok = m0 + r < M;
      const size_t off = (size_t)(ok ? m0 + r : 0) * K + k0 + col;
      cp_async16(sA + (size_t)(buf * (SPLIT ? 2 : 1)) * APL + r * TLDS + col, Ahi + off, ok);
      if constexpr (SPLIT) cp_async16(sA + (size_t)(buf * 2 + 1) * APL + r * TLDS + col, Alo + off, ok);
    }
    for (int c = tid; c < BN * 4; c += 256) {
      const int r = c >> 2, col = (c & 3) * 8;
      cp_async16(sB + (size_t)buf * BPL + r * TLDS + col, B + (size_t)(n0 + r) * K + k0 + col, true);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[MT][4][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const int nk = K / TBK;
  load(0, 0);
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nk) {
      load(kc + 1, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const __nv_bfloat16* a_hi = sA + (size_t)(buf * (SPLIT ? 2 : 1)) * APL;
    const __nv_bfloat16* b_s = sB + (size_t)buf * BPL;
#pragma unroll
    for (int kk = 0; kk < TBK; kk += 16) {
      uint32_t bf[4][2];
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const __nv_bfloat16* p = b_s + (wc + np * 16 + (lane & 7) + (lane >> 4) * 8) * TLDS + kk + ((lane >> 3) & 1) * 8;
        ldsm_x4(p, bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0], bf[2 * np + 1][1]);
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t af[4];
        const int row = wr + mt * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
        ldsm_x4(a_hi + row * TLDS + col, af[0], af[1], af[2], af[3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], af, bf[nt][0], bf[nt][1]);
        if constexpr (SPLIT) {
          ldsm_x4(a_hi + APL + row * TLDS + col, af[0], af[1], af[2], af[3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], af, bf[nt][0], bf[nt][1]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int m = m0 + wr + mt * 16 + g + (k >= 2 ? 8 : 0);
        const int n = n0 + wc + nt * 8 + 2 * q + (k & 1);
        if (m >= M) continue;
        float v = acc[mt][nt][k];
        if (e.kind == EPI_FWD_HIDDEN) {
          v = bf16_round(fmaxf(v + e.bias[n], 0.f));
          static_cast<__nv_bfloat16*>(e.out)[(size_t)m * e.ldo + n] = __float2bfloat16_rn(v);
        } else if (e.kind == EPI_BWD_HIDDEN) {
          if (!(e.mask[(size_t)(e.mask_row + n) * e.ncol + e.col0 + m] > 0.f)) v = 0.f;
          const float hi = bf16_round(v);
          static_cast<__nv_bfloat16*>(e.out)[(size_t)m * e.ldo + n] = __float2bfloat16_rn(hi);
          e.out_lo[(size_t)m * e.ldo + n] = __float2bfloat16_rn(v - hi);
        } else {
          static_cast<float*>(e.out)[(size_t)m * e.ldo + n] = v;
        }
        if (e.dump) e.dump[(size_t)(e.dump_row + n) * e.ncol + e.col0 + m] = v;
      }
}

template <int BN, bool SPLIT>
cudaError_t tc_gemm(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, const __nv_bfloat16* B, int M, int N, int K,
                    const GemmEpi& e, cudaStream_t s) {
  const int smem = (2 * (SPLIT ? 2 : 1) * TBM * TLDS + 2 * BN * TLDS) * (int)sizeof(__nv_bfloat16);
  cudaError_t r = cudaFuncSetAttribute(k_tc_gemm<BN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (r != cudaSuccess) return r;
  dim3 grid(N / BN, (M + TBM - 1) / TBM);
  k_tc_gemm<BN, SPLIT><<<grid, 256, smem, s>>>(Ahi, Alo, B, M, N, K, e);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Weight gradient of a wide layer on the tensor cores: partial[split][o][c] = sum over the split's
// dump columns n of delta[o][n] act[c][n] (Eq. 4's chain rule summed over steps and instances).
// Both operands are fp32 dump rows (column index n contiguous); they are converted to bfloat16
// while they are staged in shared memory: activations are bfloat16 values already (exact), deltas
// are split into a high and a low bfloat16 part (two products). A CTA computes a 128 x BN tile of
// rows of A against rows of B; with TRANS, A holds the activations and B the deltas (layers with
// few outputs) and the tile is stored transposed. Loads for the next 32-column chunk are issued
// into registers before the current chunk's products.
template <int BN, bool SPLIT_A, bool SPLIT_B, bool TRANS>
__global__ void __launch_bounds__(256, 2) k_dw_tc(const float* __restrict__ A, int MA, const float* __restrict__ Bm, int MB,
                                                  size_t N, size_t chunk, float* __restrict__ partial) {
  constexpr int WN = BN / 32, WM = 8 / WN, WTM = TBM / WM, MT = WTM / 16;
  constexpr int PA = SPLIT_A ? 2 : 1, PB = SPLIT_B ? 2 : 1;
  constexpr int APL = TBM * TLDS, BPL = BN * TLDS;
  constexpr int LA = TBM * 8 / 256, LB = (BN * 8 + 255) / 256;  // float4 loads per thread and chunk
  extern __shared__ __align__(16) unsigned char dw_smem[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(dw_smem);  // [2][PA][APL]
  __nv_bfloat16* sB = sA + 2 * PA * APL;                           // [2][PB][BPL]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
  const int wr = (warp / WN) * WTM, wc = (warp % WN) * 32;
  const size_t k0 = (size_t)blockIdx.z * chunk, k1 = min(N, k0 + chunk);
  const int nk = k1 > k0 ? (int)((k1 - k0) / TBK) : 0;
  float4 ra[LA], rb[LB];
  auto gload = [&](int kc) {
    const size_t kb = k0 + (size_t)kc * TBK;
#pragma unroll
    for (int j = 0; j < LA; ++j) {
      const int c = tid + j * 256, r = c >> 3, col = (c & 7) * 4;
      ra[j] = m0 + r < MA ? __ldg(reinterpret_cast<const float4*>(A + (size_t)(m0 + r) * N + kb + col))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const int c = tid + j * 256, r = c >> 3, col = (c & 7) * 4;
      rb[j] = (c < BN * 8 && n0 + r < MB) ? __ldg(reinterpret_cast<const float4*>(Bm + (size_t)(n0 + r) * N + kb + col))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto put = [](__nv_bfloat16* hi, __nv_bfloat16* lo, float4 v) {
    const float h[4] = {bf16_round(v.x), bf16_round(v.y), bf16_round(v.z), bf16_round(v.w)};
    *reinterpret_cast<uint2*>(hi) = make_uint2(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]));
    if (lo) *reinterpret_cast<uint2*>(lo) = make_uint2(pack_bf16(v.x - h[0], v.y - h[1]), pack_bf16(v.z - h[2], v.w - h[3]));
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int j = 0; j < LA; ++j) {
      const int c = tid + j * 256, r = c >> 3, col = (c & 7) * 4;
      __nv_bfloat16* p = sA + (size_t)buf * PA * APL + r * TLDS + col;
      put(p, SPLIT_A ? p + APL : nullptr, ra[j]);
    }
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const int c = tid + j * 256, r = c >> 3, col = (c & 7) * 4;
      if (c >= BN * 8) continue;
      __nv_bfloat16* p = sB + (size_t)buf * PB * BPL + r * TLDS + col;
      put(p, SPLIT_B ? p + BPL : nullptr, rb[j]);
    }
  };
  float acc[MT][4][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  if (nk > 0) {
    gload(0);
    sstore(0);
  }
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nk) gload(kc + 1);
    const __nv_bfloat16* a_s = sA + (size_t)buf * PA * APL;
    const __nv_bfloat16* b_s = sB + (size_t)buf * PB * BPL;
#pragma unroll
    for (int kk = 0; kk < TBK; kk += 16) {
      uint32_t bf[PB][4][2];
#pragma unroll
      for (int pb = 0; pb < PB; ++pb)
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          const __nv_bfloat16* p =
              b_s + pb * BPL + (wc + np * 16 + (lane & 7) + (lane >> 4) * 8) * TLDS + kk + ((lane >> 3) & 1) * 8;
          ldsm_x4(p, bf[pb][2 * np][0], bf[pb][2 * np][1], bf[pb][2 * np + 1][0], bf[pb][2 * np + 1][1]);
        }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int row = wr + mt * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
#pragma unroll
        for (int pa = 0; pa < PA; ++pa) {
          uint32_t af[4];
          ldsm_x4(a_s + pa * APL + row * TLDS + col, af[0], af[1], af[2], af[3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            mma_bf16_16816(acc[mt][nt], af, bf[0][nt][0], bf[0][nt][1]);
            if constexpr (SPLIT_B) {
              if (pa == 0) mma_bf16_16816(acc[mt][nt], af, bf[PB - 1][nt][0], bf[PB - 1][nt][1]);
            }
          }
        }
      }
    }
    if (kc + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
  float* P = partial + (size_t)blockIdx.z * MA * MB;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int m = m0 + wr + mt * 16 + g + (k >= 2 ? 8 : 0);
        const int n = n0 + wc + nt * 8 + 2 * q + (k & 1);
        if (m >= MA || n >= MB) continue;
        if (TRANS)
          P[(size_t)n * MA + m] = acc[mt][nt][k];
        else
          P[(size_t)m * MB + n] = acc[mt][nt][k];
      }
}

// Split count for a grid of `tiles` CTAs: the one whose last wave is fullest (2 CTAs per SM on
// 152 SMs), at most `cap`.
int dw_splits_for(int tiles, int cap) {
  const int slots = 2 * 152;
  int best = 1;
  double best_cost = 1e30;
  for (int s = 1; s <= std::min(cap, 64); ++s) {
    const double waves = std::ceil((double)tiles * s / slots);
    const double cost = waves / s + 1e-3 * s;  // time per unit of work, then fewer partials
    if (cost < best_cost) best_cost = cost, best = s;
  }
  return best;
}

template <int BN, bool SPLIT_A, bool SPLIT_B, bool TRANS>
cudaError_t dw_tc(const float* A, int MA, const float* Bm, int MB, size_t N, float* partial, size_t partial_floats,
                  int* splits_out, cudaStream_t s) {
  constexpr int smem = (2 * (SPLIT_A ? 2 : 1) * TBM * TLDS + 2 * (SPLIT_B ? 2 : 1) * BN * TLDS) * (int)sizeof(__nv_bfloat16);
  cudaError_t r = cudaFuncSetAttribute(k_dw_tc<BN, SPLIT_A, SPLIT_B, TRANS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (r != cudaSuccess) return r;
  const int gx = (MB + BN - 1) / BN, gy = (MA + TBM - 1) / TBM;
  const int cap = (int)std::max<size_t>(1, partial_floats / ((size_t)MA * MB));
  const int splits = dw_splits_for(gx * gy, cap);
  const size_t chunk = ((N + splits - 1) / splits + TBK - 1) / TBK * TBK;
  k_dw_tc<BN, SPLIT_A, SPLIT_B, TRANS><<<dim3(gx, gy, splits), 256, smem, s>>>(A, MA, Bm, MB, N, chunk, partial);
  *splits_out = splits;
  return cudaGetLastError();
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

// Tile width of the tiled products: 128 columns where N allows it.
template <bool SPLIT>
cudaError_t tc_gemm_n(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, const __nv_bfloat16* B, int M, int N, int K,
                      const GemmEpi& e, cudaStream_t s) {
  return N % 128 == 0 ? tc_gemm<128, SPLIT>(Ahi, Alo, B, M, N, K, e, s) : tc_gemm<64, SPLIT>(Ahi, Alo, B, M, N, K, e, s);
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
  cudaError_t r = tc_gemm_n<false>(D.s_ext, nullptr, w->ext_w + Lo.w1, M, Lo.h1, Lo.k0p, e, w->stream);
  if (r != cudaSuccess) return r;
  e.bias = D.bias + T.w_off[1];
  e.nvalid = Lo.h2;
  e.out = w->ext_h2;
  e.ldo = Lo.h2;
  e.dump_row = T.dump_act[2];
  r = tc_gemm_n<false>(w->ext_h1, nullptr, w->ext_w + Lo.w2, M, Lo.h2, Lo.h1, e, w->stream);
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
// The deltas are kept as two bfloat16 planes (high part, then the low remainder) in the fp32
// delta buffers, which hold exactly the two planes.
cudaError_t ext_backward_products(dp_world* w, const DevTopo& T, const DevPtrs& D, int t) {
  const ExtLayout& Lo = w->ext;
  const int M = T.Bp;
  __nv_bfloat16* d2 = reinterpret_cast<__nv_bfloat16*>(w->ext_d2);
  __nv_bfloat16* d1 = reinterpret_cast<__nv_bfloat16*>(w->ext_d1);
  const size_t p2 = (size_t)M * Lo.h2, p1 = (size_t)M * Lo.h1;
  GemmEpi e{};
  e.ncol = (size_t)T.horizon * T.Bp;
  e.col0 = (size_t)t * T.Bp;
  e.kind = EPI_BWD_HIDDEN;
  e.nvalid = Lo.h2;
  e.out = d2;
  e.out_lo = d2 + p2;
  e.ldo = Lo.h2;
  e.dump = D.dump;
  e.dump_row = T.dump_del[1];
  e.mask = D.dump;
  e.mask_row = T.dump_act[2];
  cudaError_t r = gemm<8, true>(D.ub_ext, 16, w->ext_w + Lo.w3t, M, Lo.h2, 16, e, w->stream);
  if (r != cudaSuccess) return r;
  e.nvalid = Lo.h1;
  e.out = d1;
  e.out_lo = d1 + p1;
  e.ldo = Lo.h1;
  e.dump_row = T.dump_del[0];
  e.mask_row = T.dump_act[1];
  r = tc_gemm_n<true>(d2, d2 + p2, w->ext_w + Lo.w2t, M, Lo.h1, Lo.h2, e, w->stream);
  if (r != cudaSuccess) return r;
  e.kind = EPI_BWD_IN;
  e.nvalid = Lo.k0p;
  e.out = const_cast<float*>(D.sbar_ext);
  e.out_lo = nullptr;
  e.ldo = Lo.k0p;
  e.dump = nullptr;
  return tc_gemm_n<true>(d1, d1 + p1, w->ext_w + Lo.w1t, M, Lo.k0p, Lo.h1, e, w->stream);
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

// Controller gradient of a 3-layer bfloat16 network on the tensor cores (the wide path, and the
// in-step tensor-core controller), summed over all steps and instances, into dst (flat layout
// of the master weights: per layer W[out][in] then b[out]). dW_l = sum over the T Bp dump columns
// of delta_l act_l^T: the activations are bfloat16 values already (exact), the fp32 deltas enter
// as two bfloat16 parts (hi + lo, 16 significant bits).
cudaError_t tc_weight_grad(dp_world* w, const DevTopo& T, const DevPtrs& D, float* dst) {
  const size_t N = (size_t)T.horizon * T.Bp;
  const int rows[4] = {T.widths[0], T.widths[1], T.widths[2], T.widths[3]};
  size_t off = 0;
  for (int l = 0; l < 3; ++l) {
    const int ni = rows[l], no_ = rows[l + 1];
    const float* del = D.dump + (size_t)T.dump_del[l] * N;
    const float* act = D.dump + (size_t)T.dump_act[l] * N;
    int splits = 1;
    cudaError_t r;
    if (l == 2)
      r = dw_tc<32, false, true, true>(act, ni, del, no_, N, w->partial, w->partial_floats, &splits, w->stream);
    else if (ni <= 64)
      r = dw_tc<64, true, false, false>(del, no_, act, ni, N, w->partial, w->partial_floats, &splits, w->stream);
    else
      r = dw_tc<128, true, false, false>(del, no_, act, ni, N, w->partial, w->partial_floats, &splits, w->stream);
    if (r == cudaSuccess) r = launch_sum_splits(w->partial, splits, (size_t)no_ * ni, dst + off, w->stream);
    if (r != cudaSuccess) return r;
    off += (size_t)no_ * ni;
    const int bs = w->splits;
    const size_t chunk = ((N + bs - 1) / bs + 15) / 16 * 16;
    r = launch_rowsum(del, no_, N, w->partial, bs, chunk, w->stream);
    if (r == cudaSuccess) r = launch_sum_splits(w->partial, bs, (size_t)no_, dst + off, w->stream);
    if (r != cudaSuccess) return r;
    off += no_;
  }
  return cudaSuccess;
}
