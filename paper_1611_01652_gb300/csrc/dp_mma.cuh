// Warp-level dense networks on the BF16 tensor cores (mma.sync m16n8k16, fp32 accumulate) for
// the lane-per-instance layout: the rows of a layer's input are the lanes of a [feature][32]
// shared-memory array, processed one 16-row m-tile at a time. A hidden layer's output fragments
// are converted in registers into the next layer's input fragments, so hidden activations never
// leave the register file. Reverse mode splits each fp32 adjoint into two bfloat16 parts
// (hi + lo) so that the products keep about 16 significant bits.
//
// Fragment layout of m16n8k16 (PTX ISA, "Matrix Fragments for mma.m16n8k16"): with g = lane / 4
// and q = lane % 4, A (16x16, row-major) a0 = (g, 2q..2q+1), a1 = (g+8, 2q..), a2 = (g, 2q+8..),
// a3 = (g+8, 2q+8..); B (16x8, column-major) b0 = (k = 2q..2q+1, n = g), b1 = (k = 2q+8.., n = g);
// C (16x8) c0 = (g, 2q), c1 = (g, 2q+1), c2 = (g+8, 2q), c3 = (g+8, 2q+1).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <int N>
__device__ __forceinline__ constexpr int pad16() { return (N + 15) / 16 * 16; }
template <int N>
__device__ __forceinline__ constexpr int pad8() { return (N + 7) / 8 * 8; }

// B fragments of W (stored [n][Kp] bf16, k contiguous): columns n0 + g, rows k0 + 2q (+8).
__device__ __forceinline__ void load_b(const __nv_bfloat16* __restrict__ W, int Kp, int n0, int k0, uint32_t& b0,
                                       uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const __nv_bfloat16* p = W + (size_t)(n0 + g) * Kp + k0 + 2 * q;
  b0 = __ldg(reinterpret_cast<const unsigned int*>(p));
  b1 = __ldg(reinterpret_cast<const unsigned int*>(p + 8));
}

// A fragments of one k-tile of the input x(f, row) (rows of m-tile mt; features >= K are zero).
template <int K, class IN>
__device__ __forceinline__ void load_a_lanes(IN& x, int mt, int kt, uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8, c = kt * 16 + 2 * q;
  auto v = [&](int f, int r) { return f < K ? x(f, r) : 0.f; };
  a[0] = pack_bf16(v(c, r0), v(c + 1, r0));
  a[1] = pack_bf16(v(c, r1), v(c + 1, r1));
  a[2] = pack_bf16(v(c + 8, r0), v(c + 9, r0));
  a[3] = pack_bf16(v(c + 8, r1), v(c + 9, r1));
}

// One dense layer on an m-tile: acc[NT][4] = bias + A (KT k-tiles) * W^T. W is [Np][Kp] bf16.
template <int KT, int NT>
__device__ __forceinline__ void dense_mma(const uint32_t (&a)[KT][4], const __nv_bfloat16* __restrict__ W,
                                          const float* __restrict__ bias, int nvalid, float (&acc)[NT][4]) {
  const int q = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = nt * 8 + 2 * q;
    const float b0 = bias && c < nvalid ? __ldg(bias + c) : 0.f;
    const float b1 = bias && c + 1 < nvalid ? __ldg(bias + c + 1) : 0.f;
    acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
  }
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      load_b(W, KT * 16, nt * 8, kt * 16, b0, b1);
      mma_bf16_16816(acc[nt], a[kt], b0, b1);
    }
}

// ReLU, bfloat16 rounding, and the C -> A fragment conversion for the next layer.
template <int NT>
__device__ __forceinline__ void relu_to_a(float (&acc)[NT][4], uint32_t (&a)[NT / 2][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[nt][k] = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[nt][k], 0.f)));
#pragma unroll
  for (int kt = 0; kt < NT / 2; ++kt) {
    a[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
    a[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
    a[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
    a[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
  }
}

// Store C fragments (features along n) of an m-tile: dst(f, row) = acc.
template <int NT, class F>
__device__ __forceinline__ void store_c(const float (&acc)[NT][4], int mt, int nvalid, F&& dst) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = nt * 8 + 2 * q;
    if (c < nvalid) { dst(c, r0, acc[nt][0]); dst(c, r1, acc[nt][2]); }
    if (c + 1 < nvalid) { dst(c + 1, r0, acc[nt][1]); dst(c + 1, r1, acc[nt][3]); }
  }
}

// bfloat16 weight layouts of the 24-128-128-8 controller for the tensor-core path: forward
// matrices [out][in_pad16] and transposed matrices [in][out_pad16] (padding is zero).
struct CtrlTC {
  static constexpr int K0 = 24, H1 = 128, H2 = 128, NO = 8;
  static constexpr int W1 = 0;                   // [H1][32]
  static constexpr int W2 = W1 + H1 * 32;        // [H2][H1]
  static constexpr int W3 = W2 + H2 * H1;        // [8][H2]
  static constexpr int W3T = W3 + 8 * H2;        // [H2][16]
  static constexpr int W2T = W3T + H2 * 16;      // [H1][H2]
  static constexpr int W1T = W2T + H1 * H2;      // [24][H1]
  static constexpr int SIZE = W1T + 24 * H1;
};

// The learned warm-start network 16-64-64-3: bfloat16 tensor-core layouts (as CtrlTC) and the
// fp32 bias array; the flat fp32 parameter vector is W1[64][16], b1, W2[64][64], b2, W3[3][64], b3.
struct WsTC {
  static constexpr int K0 = 16, H1 = 64, H2 = 64, NO = 3;
  static constexpr int W1 = 0;                   // [H1][16]
  static constexpr int W2 = W1 + H1 * 16;        // [H2][H1]
  static constexpr int W3 = W2 + H2 * H1;        // [8][H2]
  static constexpr int W3T = W3 + 8 * H2;        // [H2][16]
  static constexpr int W2T = W3T + H2 * 16;      // [H1][H2]
  static constexpr int W1T = W2T + H1 * H2;      // [16][H1]
  static constexpr int SIZE = W1T + 16 * H1;
  static constexpr int B1 = 0, B2 = 64, B3 = 128, BSIZE = 136;
  // flat parameter offsets
  static constexpr int F_W1 = 0, F_B1 = F_W1 + H1 * K0, F_W2 = F_B1 + H1, F_B2 = F_W2 + H2 * H1, F_W3 = F_B2 + H2,
                       F_B3 = F_W3 + NO * H2, PARAMS = F_B3 + NO;
};

// Three dense layers K0 -> H1 -> H2 -> NO (ReLU hidden, linear output) for the 32 rows of a
// warp. in(f, row): the K0 inputs (bfloat16-exact fp32); weights [Np][Kp] bf16 with fp32 biases;
// out(f, row, v) receives the NO outputs; hid(layer, f, row, v) the hidden activations.
template <int K0, int H1, int H2, int NO, class IN, class OUT, class HID>
__device__ void mlp3_forward(IN&& in, const __nv_bfloat16* W1, const float* b1, const __nv_bfloat16* W2,
                             const float* b2, const __nv_bfloat16* W3, const float* b3, OUT&& out, HID&& hid) {
  constexpr int KT0 = pad16<K0>() / 16, NT1 = H1 / 8, NT2 = H2 / 8, NT3 = pad8<NO>() / 8;
  static_assert(H1 % 16 == 0 && H2 % 16 == 0, "hidden widths must be multiples of 16");
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a0[KT0][4];
#pragma unroll
    for (int kt = 0; kt < KT0; ++kt) load_a_lanes<K0>(in, mt, kt, a0[kt]);
    uint32_t a1[NT1 / 2][4];
    {
      float acc[NT1][4];
      dense_mma<KT0, NT1>(a0, W1, b1, H1, acc);
      relu_to_a<NT1>(acc, a1);
      store_c<NT1>(acc, mt, H1, [&](int f, int r, float v) { hid(1, f, r, v); });
    }
    uint32_t a2[NT2 / 2][4];
    {
      float acc[NT2][4];
      dense_mma<NT1 / 2, NT2>(a1, W2, b2, H2, acc);
      relu_to_a<NT2>(acc, a2);
      store_c<NT2>(acc, mt, H2, [&](int f, int r, float v) { hid(2, f, r, v); });
    }
    float acc[NT3][4];
    dense_mma<NT2 / 2, NT3>(a2, W3, b3, NO, acc);
    store_c<NT3>(acc, mt, NO, out);
  }
}

// hi/lo bfloat16 split of an fp32 C fragment array into A fragments.
template <int NT>
__device__ __forceinline__ void split_to_a(const float (&d)[NT][4], uint32_t (&hi)[NT / 2][4], uint32_t (&lo)[NT / 2][4]) {
#pragma unroll
  for (int kt = 0; kt < NT / 2; ++kt) {
    const float* x0 = d[2 * kt];
    const float* x1 = d[2 * kt + 1];
    float h[8], l[8];
    const float v[8] = {x0[0], x0[1], x0[2], x0[3], x1[0], x1[1], x1[2], x1[3]};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      h[k] = __bfloat162float(__float2bfloat16_rn(v[k]));
      l[k] = v[k] - h[k];
    }
    hi[kt][0] = pack_bf16(h[0], h[1]); hi[kt][1] = pack_bf16(h[2], h[3]);
    hi[kt][2] = pack_bf16(h[4], h[5]); hi[kt][3] = pack_bf16(h[6], h[7]);
    lo[kt][0] = pack_bf16(l[0], l[1]); lo[kt][1] = pack_bf16(l[2], l[3]);
    lo[kt][2] = pack_bf16(l[4], l[5]); lo[kt][3] = pack_bf16(l[6], l[7]);
  }
}

// acc[NT][4] += (hi + lo) * W'^T with W' stored [Np][Kp] bf16 (here the transposed weights).
template <int KT, int NT>
__device__ __forceinline__ void dense_mma_split(const uint32_t (&hi)[KT][4], const uint32_t (&lo)[KT][4],
                                                const __nv_bfloat16* __restrict__ W, float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      load_b(W, KT * 16, nt * 8, kt * 16, b0, b1);
      mma_bf16_16816(acc[nt], hi[kt], b0, b1);
      mma_bf16_16816(acc[nt], lo[kt], b0, b1);
    }
}

// Reverse mode of mlp3_forward for the 32 rows of a warp. ubar(f, row): the output adjoint. mask(layer, f, row) tells whether hidden unit f of that layer was positive.
// del(layer, f, row, v) receives the adjoint of each layer's pre-activation output (layer 3 =
// output, 2, 1 hidden); sbar(f, row, v) the input adjoint. Transposed weights W't are [Kin_p][Kout_p].
template <int K0, int H1, int H2, int NO, class UBAR, class MASK, class DEL, class SBAR>
__device__ void mlp3_backward(UBAR&& ubar, const __nv_bfloat16* W3t, const __nv_bfloat16* W2t,
                              const __nv_bfloat16* W1t, MASK&& mask, DEL&& del, SBAR&& sbar) {
  constexpr int NT2 = H2 / 8, NT1 = H1 / 8, NT0 = pad8<K0>() / 8;
  constexpr int KT3 = pad16<NO>() / 16;
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // output adjoint (fp32) -> hi/lo A fragments
    uint32_t h3[KT3][4], l3[KT3][4];
    {
      float d3[2 * KT3][4];
#pragma unroll
      for (int nt = 0; nt < 2 * KT3; ++nt) {
        const int c = nt * 8 + 2 * q, r0 = mt * 16 + g, r1 = r0 + 8;
        d3[nt][0] = c < NO ? ubar(c, r0) : 0.f;
        d3[nt][1] = c + 1 < NO ? ubar(c + 1, r0) : 0.f;
        d3[nt][2] = c < NO ? ubar(c, r1) : 0.f;
        d3[nt][3] = c + 1 < NO ? ubar(c + 1, r1) : 0.f;
      }
      split_to_a<2 * KT3>(d3, h3, l3);
    }
    uint32_t h2[NT2 / 2][4], l2[NT2 / 2][4];
    {
      float d2[NT2][4];
      dense_mma_split<KT3, NT2>(h3, l3, W3t, d2);
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) {
        const int c = nt * 8 + 2 * q, r0 = mt * 16 + g, r1 = r0 + 8;
        if (!mask(2, c, r0)) d2[nt][0] = 0.f;
        if (!mask(2, c + 1, r0)) d2[nt][1] = 0.f;
        if (!mask(2, c, r1)) d2[nt][2] = 0.f;
        if (!mask(2, c + 1, r1)) d2[nt][3] = 0.f;
      }
      store_c<NT2>(d2, mt, H2, [&](int f, int r, float v) { del(2, f, r, v); });
      split_to_a<NT2>(d2, h2, l2);
    }
    uint32_t h1[NT1 / 2][4], l1[NT1 / 2][4];
    {
      float d1[NT1][4];
      dense_mma_split<NT2 / 2, NT1>(h2, l2, W2t, d1);
#pragma unroll
      for (int nt = 0; nt < NT1; ++nt) {
        const int c = nt * 8 + 2 * q, r0 = mt * 16 + g, r1 = r0 + 8;
        if (!mask(1, c, r0)) d1[nt][0] = 0.f;
        if (!mask(1, c + 1, r0)) d1[nt][1] = 0.f;
        if (!mask(1, c, r1)) d1[nt][2] = 0.f;
        if (!mask(1, c + 1, r1)) d1[nt][3] = 0.f;
      }
      store_c<NT1>(d1, mt, H1, [&](int f, int r, float v) { del(1, f, r, v); });
      split_to_a<NT1>(d1, h1, l1);
    }
    float s[NT0][4];
    dense_mma_split<NT1 / 2, NT0>(h1, l1, W1t, s);
    store_c<NT0>(s, mt, K0, sbar);
  }
}
