// Kernels of libdphys around the rollout: weight staging, layout transposes, the gradient check
// and the controller-gradient reduction. The persistent rollout and reverse-mode kernels are in
// dp_steps.cuh, instantiated by dp_fwd.cu, dp_bwd.cu, dp_bwd_mw.cu and dp_bwd_ext.cu (one
// translation unit per kernel family, so that they compile in parallel).
#include <cuda_runtime.h>

#include "dp_static.cuh"
#include "dp_kernels.h"

// ------------------------------------------------------------------------------ weights
// Flat fp32 master weights -> bf16-rounded fp32 copies in two layouts, fp32 biases.
__global__ void k_prep_weights(const __grid_constant__ DevTopo T, const float* __restrict__ W, float* Wt, float* Wn,
                               float* bias) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.n_params) return;
  int off = 0;
  const int nl = T.n_layers + (T.skip ? 1 : 0);
  for (int l = 0; l < nl; ++l) {
    const int ni = l < T.n_layers ? T.widths[l] : T.widths[0];
    const int no = l < T.n_layers ? T.widths[l + 1] : T.widths[T.n_layers];
    const int nop = (no + 7) & ~7, nip = (ni + 7) & ~7;
    if (p < off + ni * no) {
      int q = p - off, o = q / ni, i = q % ni;
      float w = T.ctrl_round ? bf16r(W[p]) : W[p];
      Wt[T.w_off[l] + i * nop + o] = w;
      Wn[T.w_off[l] + o * nip + i] = w;
      return;
    }
    off += ni * no;
    if (p < off + no) {
      bias[T.w_off[l] + (p - off)] = W[p];
      return;
    }
    off += no;
  }
}

// Tensor-core layouts of a K0-H1-H2-NO controller (ctrl_tc_layout), bfloat16, zero padded.
__global__ void k_prep_weights_tc(const __grid_constant__ DevTopo T, const float* __restrict__ W, __nv_bfloat16* Wc) {
  const int K0 = T.widths[0], H1 = T.widths[1], H2 = T.widths[2], NO = T.widths[3];
  const CtrlTCLayout Lw = ctrl_tc_layout(H1, H2);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Lw.size) return;
  // flat master layout: per layer W[out][in] then b[out]
  const int m1 = K0 * H1 + H1, m2 = m1 + H1 * H2 + H2;
  auto w = [&](int l, int o, int i) { return W[(l == 0 ? 0 : l == 1 ? m1 : m2) + o * T.widths[l] + i]; };
  float v = 0.f;
  if (p < Lw.w2) {  // W1 [H1][32]
    const int o = p / CTRL_TC_KP0, i = p % CTRL_TC_KP0;
    v = i < K0 ? w(0, o, i) : 0.f;
  } else if (p < Lw.w3) {  // W2 [H2][H1]
    const int q = p - Lw.w2, o = q / H1, i = q % H1;
    v = w(1, o, i);
  } else if (p < Lw.w3t) {  // W3 [16][H2]
    const int q = p - Lw.w3, o = q / H2, i = q % H2;
    v = o < NO ? w(2, o, i) : 0.f;
  } else if (p < Lw.w2t) {  // W3^T [H2][16]
    const int q = p - Lw.w3t, i = q / CTRL_TC_NOP, o = q % CTRL_TC_NOP;
    v = o < NO ? w(2, o, i) : 0.f;
  } else if (p < Lw.w1t) {  // W2^T [H1][H2]
    const int q = p - Lw.w2t, i = q / H2, o = q % H2;
    v = w(1, o, i);
  } else {  // W1^T [32][H1]
    const int q = p - Lw.w1t, i = q / H1, o = q % H1;
    v = i < K0 ? w(0, o, i) : 0.f;
  }
  Wc[p] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------------------ layouts
// [B][nb*18] (user) -> [nb*18][Bp]; padded instances copy instance B-1.
__global__ void k_state_in(int B, int Bp, int nf, const float* __restrict__ src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp) return;
  int si = i < B ? i : B - 1;
  for (int f = 0; f < nf; ++f) dst[(size_t)f * Bp + i] = src[(size_t)si * nf + f];
}
__global__ void k_state_out(int B, int Bp, int nf, const float* __restrict__ src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  for (int f = 0; f < nf; ++f) dst[(size_t)i * nf + f] = src[(size_t)f * Bp + i];
}
// Gather one parameter group: user [B][n] <-> internal field offset o, n fields.
__global__ void k_param_out(int B, int Bp, int o, int n, const float* __restrict__ src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  for (int f = 0; f < n; ++f) dst[(size_t)i * n + f] = src[(size_t)(o + f) * Bp + i];
}
// Per-instance parameter group [B][n] -> the [field][Bp] parameter array (padded lanes copy the
// last instance).
__global__ void k_param_in(int B, int Bp, int o, int n, const float* __restrict__ src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp) return;
  const int si = min(i, B - 1);
  for (int f = 0; f < n; ++f) dst[(size_t)(o + f) * Bp + i] = src[(size_t)si * n + f];
}
__global__ void k_scale_out(int B, const float* __restrict__ src, float sc, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) dst[i] = src[i] * sc;
}
__global__ void k_pad_scalar(int B, int Bp, const float* __restrict__ src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp) return;
  dst[i] = i < B ? src[i] : 0.f;
}

__global__ void k_check_grads(int B, int Bp, int nf, int np, const float* __restrict__ gs, const float* __restrict__ gp,
                              int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  bool bad = false;
  for (int f = 0; f < nf; ++f) bad |= !isfinite(gs[(size_t)f * Bp + i]);
  for (int f = 0; f < np; ++f) bad |= !isfinite(gp[(size_t)f * Bp + i]);
  status[i] = (status[i] & ~DPK_ST_NAN_GRAD) | (bad ? DPK_ST_NAN_GRAD : 0);
}
cudaError_t launch_check_grads(int B, int Bp, int nf, int np, const float* gs, const float* gp, int* status,
                               cudaStream_t s) {
  k_check_grads<<<(B + 127) / 128, 128, 0, s>>>(B, Bp, nf, np, gs, gp, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ dW reduction
// partial[split][o][c] = sum over columns n in the split of del[o][n] * act[c][n]
// (64x64 output tile per block, 256 threads, 4x4 outputs per thread).
__global__ void __launch_bounds__(256) k_dw_gemm(const float* __restrict__ del, const float* __restrict__ act, int M,
                                                 int C, size_t N, size_t chunk, float* __restrict__ partial) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int o0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const size_t n0 = (size_t)blockIdx.z * chunk;
  const size_t n1 = min(N, n0 + chunk);
  float acc[4][4] = {};
  for (size_t nb = n0; nb < n1; nb += 16) {
    // load 64 rows x 16 columns of each operand (coalesced along n)
    for (int q = threadIdx.x; q < 64 * 16; q += 256) {
      int r = q / 16, k = q % 16;
      size_t n = nb + k;
      As[k][r] = (o0 + r < M && n < n1) ? del[(size_t)(o0 + r) * N + n] : 0.f;
      Bs[k][r] = (c0 + r < C && n < n1) ? act[(size_t)(c0 + r) * N + n] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[k][ty * 4 + u]; b[u] = Bs[k][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float* P = partial + (size_t)blockIdx.z * M * C;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int o = o0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (o < M && c < C) P[(size_t)o * C + c] = acc[u][v];
    }
}
// partial[split][o] = sum over the split's columns of del[o][n]
__global__ void k_rowsum(const float* __restrict__ del, int M, size_t N, size_t chunk, float* __restrict__ partial) {
  const int o = blockIdx.y;
  const size_t n0 = (size_t)blockIdx.x * chunk, n1 = min(N, n0 + chunk);
  float s = 0.f;
  for (size_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) s += del[(size_t)o * N + n];
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * M + o] = red[0];
}
// out[k] = sum over splits of partial[split][k] (fixed order: deterministic)
__global__ void k_sum_splits(const float* __restrict__ partial, int splits, size_t count, float* __restrict__ out) {
  size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  float s = 0.f;
  for (int q = 0; q < splits; ++q) s += partial[(size_t)q * count + k];
  out[k] = s;
}

// ------------------------------------------------------------------------------ launchers

cudaError_t launch_prep_weights(const DevTopo& T, const float* W, float* Wt, float* Wn, float* bias, cudaStream_t s) {
  if (T.n_params == 0) return cudaSuccess;
  k_prep_weights<<<(T.n_params + 255) / 256, 256, 0, s>>>(T, W, Wt, Wn, bias);
  return cudaGetLastError();
}
cudaError_t launch_prep_weights_tc(const DevTopo& T, const float* W, __nv_bfloat16* Wc, cudaStream_t s) {
  const int n = ctrl_tc_layout(T.widths[1], T.widths[2]).size;
  k_prep_weights_tc<<<(n + 255) / 256, 256, 0, s>>>(T, W, Wc);
  return cudaGetLastError();
}
cudaError_t launch_state_in(int B, int Bp, int nf, const float* src, float* dst, cudaStream_t s) {
  k_state_in<<<(Bp + 127) / 128, 128, 0, s>>>(B, Bp, nf, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_state_out(int B, int Bp, int nf, const float* src, float* dst, cudaStream_t s) {
  k_state_out<<<(B + 127) / 128, 128, 0, s>>>(B, Bp, nf, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_param_out(int B, int Bp, int o, int n, const float* src, float* dst, cudaStream_t s) {
  k_param_out<<<(B + 127) / 128, 128, 0, s>>>(B, Bp, o, n, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_param_in(int B, int Bp, int o, int n, const float* src, float* dst, cudaStream_t s) {
  k_param_in<<<(Bp + 127) / 128, 128, 0, s>>>(B, Bp, o, n, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_scale_out(int B, const float* src, float scale, float* dst, cudaStream_t s) {
  k_scale_out<<<(B + 127) / 128, 128, 0, s>>>(B, src, scale, dst);
  return cudaGetLastError();
}
cudaError_t launch_pad_scalar(int B, int Bp, const float* src, float* dst, cudaStream_t s) {
  k_pad_scalar<<<(Bp + 127) / 128, 128, 0, s>>>(B, Bp, src, dst);
  return cudaGetLastError();
}
// Compiled topology Q matching a run-time one: its id, or 0. The compiled schedule must also
// equal the run-time schedule slot for slot.
template <class Q>
static int match_one(const DevTopo& T, int nb, int nj, int ns, int np, const int* jtype, const int* jbody,
                     const int* jflags, const int* sbody, const int* pair) {
  if (!topo_matches<Q>(nb, nj, ns, np, jtype, jbody, jflags, sbody, pair)) return 0;
  const SlotTab& S = Q::S;
  if (S.n != T.nslots) return 0;
  for (int q = 0; q < S.n; ++q)
    if (S.kind[q] != T.skind[q] || S.a[q] != T.sa[q] || S.b[q] != T.sb[q] || S.order[q] != T.order[q] ||
        S.normal[q] != T.snormal[q] || S.sub[q] != T.ssub[q] || S.idx[q] != T.sidx[q])
      return 0;
  return Q::id;
}
int match_compiled_topology(const DevTopo& T, int nb, int nj, int ns, int np, const int* jtype, const int* jbody,
                            const int* jflags, const int* sbody, const int* pair) {
  int id = match_one<QuadrupedTopo>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  if (!id) id = match_one<ArmTopo<3>>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  if (!id) id = match_one<ArmTopo<4>>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  if (!id) id = match_one<ArmTopo<5>>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  if (!id) id = match_one<ArmTopo<6>>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  if (!id) id = match_one<ArmTopo<7>>(T, nb, nj, ns, np, jtype, jbody, jflags, sbody, pair);
  return id;
}
int compiled_ctrl_width(int topo_id) {
  if (topo_id == QuadrupedTopo::id) return QuadrupedTopo::CTRL_H;
  if (topo_id >= ArmTopo<3>::id && topo_id <= ArmTopo<7>::id) return ArmTopo<3>::CTRL_H;
  return 0;
}
cudaError_t launch_dw(const float* del, const float* act, int M, int C, size_t N, float* partial, int splits,
                      size_t chunk, cudaStream_t s) {
  dim3 g((C + 63) / 64, (M + 63) / 64, splits);
  k_dw_gemm<<<g, 256, 0, s>>>(del, act, M, C, N, chunk, partial);
  return cudaGetLastError();
}
cudaError_t launch_rowsum(const float* del, int M, size_t N, float* partial, int splits, size_t chunk, cudaStream_t s) {
  dim3 g(splits, M);
  k_rowsum<<<g, 256, 0, s>>>(del, M, N, chunk, partial);
  return cudaGetLastError();
}
cudaError_t launch_sum_splits(const float* partial, int splits, size_t count, float* out, cudaStream_t s) {
  k_sum_splits<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(partial, splits, count, out);
  return cudaGetLastError();
}
