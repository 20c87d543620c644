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

// A fragments of one k-tile of the input x(f, row) (rows of m-tile mt; features >= k0 are zero).
template <class IN>
__device__ __forceinline__ void load_a_lanes(IN& x, int k0, int mt, int kt, uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8, c = kt * 16 + 2 * q;
  auto v = [&](int f, int r) { return f < k0 ? x(f, r) : 0.f; };
  a[0] = pack_bf16(v(c, r0), v(c + 1, r0));
  a[1] = pack_bf16(v(c, r1), v(c + 1, r1));
  a[2] = pack_bf16(v(c + 8, r0), v(c + 9, r0));
  a[3] = pack_bf16(v(c + 8, r1), v(c + 9, r1));
}

// acc[NT][4] += A (KT k-tiles, the matrix's k-tiles k1 / 16 ..) * W^T for the output columns
// n1 .. n1 + 8 NT. W is [N][Kp] bf16 (k contiguous).
template <int KT, int NT>
__device__ __forceinline__ void mma_acc(const uint32_t (&a)[KT][4], const __nv_bfloat16* __restrict__ W, int Kp, int n1,
                                        int k1, float (&acc)[NT][4]) {
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      load_b(W, Kp, n1 + nt * 8, k1 + kt * 16, b0, b1);
      mma_bf16_16816(acc[nt], a[kt], b0, b1);
    }
}

// acc[NT][4] = bias + A * W^T for the output columns n1 .. n1 + 8 NT (columns >= nvalid get no bias).
template <int NT>
__device__ __forceinline__ void bias_init(const float* __restrict__ bias, int n1, int nvalid, float (&acc)[NT][4]) {
  const int q = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = n1 + nt * 8 + 2 * q;
    const float b0 = bias && c < nvalid ? __ldg(bias + c) : 0.f;
    const float b1 = bias && c + 1 < nvalid ? __ldg(bias + c + 1) : 0.f;
    acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
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

// Store C fragments (features along n, the first at column n1) of an m-tile: dst(f, row) = acc.
template <int NT, class F>
__device__ __forceinline__ void store_c(const float (&acc)[NT][4], int mt, int n1, int nvalid, F&& dst) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = n1 + nt * 8 + 2 * q;
    if (c < nvalid) { dst(c, r0, acc[nt][0]); dst(c, r1, acc[nt][2]); }
    if (c + 1 < nvalid) { dst(c + 1, r0, acc[nt][1]); dst(c + 1, r1, acc[nt][3]); }
  }
}

// bfloat16 weight layouts of an in-step controller K0-H1-H2-NO on the tensor cores (K0 <= 32
// inputs, NO <= 16 outputs, hidden widths multiples of 64): forward matrices [out][in_pad] and
// transposed matrices [in][out_pad], padding zero. Offsets in bfloat16 elements.
struct CtrlTCLayout {
  int w1, w2, w3, w3t, w2t, w1t, size;
};
__host__ __device__ constexpr CtrlTCLayout ctrl_tc_layout(int h1, int h2) {
  CtrlTCLayout l{};
  l.w1 = 0;                   // [H1][32]
  l.w2 = l.w1 + h1 * 32;      // [H2][H1]
  l.w3 = l.w2 + h2 * h1;      // [16][H2]
  l.w3t = l.w3 + 16 * h2;     // [H2][16]
  l.w2t = l.w3t + h2 * 16;    // [H1][H2]
  l.w1t = l.w2t + h1 * h2;    // [32][H1]
  l.size = l.w1t + 32 * h1;
  return l;
}
constexpr int CTRL_TC_KP0 = 32, CTRL_TC_NOP = 16;
// Hidden widths with a compiled tensor-core controller (both layers the same width).
__host__ __device__ constexpr bool ctrl_tc_width(int h) { return h == 64 || h == 128 || h == 256; }

// The learned warm-start network 16-64-64-3: bfloat16 tensor-core layouts (as the controller's) and the
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

// Hidden layers are computed in chunks of MMA_CHUNK output columns, so that a layer's
// accumulators never hold more than one chunk (a 256-wide layer fits the register file).
#define MMA_CHUNK 64

// Three dense layers k0 -> H1 -> H2 -> no (ReLU hidden, linear output) for the 32 rows of a
// warp, k0 <= KP0 inputs and no <= NOP outputs. in(f, row): the inputs (bfloat16-exact fp32);
// weights [N][Kp] bf16 with fp32 biases; out(f, row, v) receives the outputs; hid(layer, f,
// row, v) the hidden activations. Layer 2's chunks feed layer 3's accumulators directly. Every
// output's sum runs over k in increasing order, whatever the chunking. Only the 16-row m-tiles
// mt0 .. mt1 - 1 are computed (two warps may take one each).
template <int KP0, int H1, int H2, int NOP, class IN, class OUT, class HID>
__device__ void mlp3_forward(int k0, int no, IN&& in, const __nv_bfloat16* W1, const float* b1, const __nv_bfloat16* W2,
                             const float* b2, const __nv_bfloat16* W3, const float* b3, OUT&& out, HID&& hid,
                             int mt0 = 0, int mt1 = 2) {
  constexpr int KT0 = pad16<KP0>() / 16, NT3 = pad8<NOP>() / 8, C = MMA_CHUNK, NTC = C / 8;
  static_assert(H1 % C == 0 && H2 % C == 0, "hidden widths must be multiples of the chunk");
#pragma unroll 1
  for (int mt = mt0; mt < mt1; ++mt) {
    uint32_t a0[KT0][4];
#pragma unroll
    for (int kt = 0; kt < KT0; ++kt) load_a_lanes(in, k0, mt, kt, a0[kt]);
    uint32_t a1[H1 / 16][4];
#pragma unroll
    for (int c = 0; c < H1 / C; ++c) {
      float acc[NTC][4];
      bias_init<NTC>(b1, c * C, H1, acc);
      mma_acc<KT0, NTC>(a0, W1, KT0 * 16, c * C, 0, acc);
      uint32_t t[NTC / 2][4];
      relu_to_a<NTC>(acc, t);
      store_c<NTC>(acc, mt, c * C, H1, [&](int f, int r, float v) { hid(1, f, r, v); });
#pragma unroll
      for (int kt = 0; kt < NTC / 2; ++kt)
#pragma unroll
        for (int e = 0; e < 4; ++e) a1[c * (NTC / 2) + kt][e] = t[kt][e];
    }
    float acc3[NT3][4];
    bias_init<NT3>(b3, 0, no, acc3);
#pragma unroll
    for (int c = 0; c < H2 / C; ++c) {
      float acc[NTC][4];
      bias_init<NTC>(b2, c * C, H2, acc);
      mma_acc<H1 / 16, NTC>(a1, W2, H1, c * C, 0, acc);
      uint32_t a2[NTC / 2][4];
      relu_to_a<NTC>(acc, a2);
      store_c<NTC>(acc, mt, c * C, H2, [&](int f, int r, float v) { hid(2, f, r, v); });
      mma_acc<NTC / 2, NT3>(a2, W3, H2, 0, c * C, acc3);
    }
    store_c<NT3>(acc3, mt, 0, no, out);
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

// acc[NT][4] += (hi + lo) * W'^T for the output columns n1 .. n1 + 8 NT, the k-tiles from k1;
// W' stored [N][Kp] bf16 (here the transposed weights).
template <int KT, int NT>
__device__ __forceinline__ void mma_acc_split(const uint32_t (&hi)[KT][4], const uint32_t (&lo)[KT][4],
                                              const __nv_bfloat16* __restrict__ W, int Kp, int n1, int k1,
                                              float (&acc)[NT][4]) {
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      load_b(W, Kp, n1 + nt * 8, k1 + kt * 16, b0, b1);
      mma_bf16_16816(acc[nt], hi[kt], b0, b1);
      mma_bf16_16816(acc[nt], lo[kt], b0, b1);
    }
}
template <int NT>
__device__ __forceinline__ void zero_acc(float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
}
// Zeroes the fragment entries of hidden layer l whose unit was not positive (ReLU adjoint).
template <int NT, class MASK>
__device__ __forceinline__ void relu_mask(float (&d)[NT][4], MASK& mask, int l, int mt, int n1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = n1 + nt * 8 + 2 * q;
    if (!mask(l, c, r0)) d[nt][0] = 0.f;
    if (!mask(l, c + 1, r0)) d[nt][1] = 0.f;
    if (!mask(l, c, r1)) d[nt][2] = 0.f;
    if (!mask(l, c + 1, r1)) d[nt][3] = 0.f;
  }
}

// Reverse mode of mlp3_forward for the 32 rows of a warp. ubar(f, row): the output adjoint
// (no <= NOP outputs); mask(layer, f, row): whether hidden unit f of that layer was positive;
// del(layer, f, row, v) receives the adjoint of each hidden layer's pre-activation (2, 1);
// sbar(f, row, v) the adjoint of the k0 inputs. Transposed weights W't are [Kin_p][Kout_p]. The
// first layer's deltas are formed C1 = min(H1, 128) columns at a time, each from every
// MMA_CHUNK-column chunk of the second layer's deltas (recomputed when H1 > 128: their product
// has only NOP terms), so that a 256-wide network's deltas are never held whole; every sum still
// runs over k in increasing order. Only the 16-row m-tiles mt0 .. mt1 - 1 are computed.
template <int KP0, int H1, int H2, int NOP, class UBAR, class MASK, class DEL, class SBAR>
__device__ void mlp3_backward(int k0, int no, UBAR&& ubar, const __nv_bfloat16* W3t, const __nv_bfloat16* W2t,
                              const __nv_bfloat16* W1t, MASK&& mask, DEL&& del, SBAR&& sbar, int mt0 = 0, int mt1 = 2) {
  constexpr int NT0 = pad8<KP0>() / 8, KT3 = pad16<NOP>() / 16, C = MMA_CHUNK, NTC = C / 8;
  constexpr int C1 = H1 < 128 ? H1 : 128, NT1 = C1 / 8;
  static_assert(H1 % C1 == 0 && H2 % C == 0 && C1 % 16 == 0, "hidden widths must be multiples of the chunks");
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll 1
  for (int mt = mt0; mt < mt1; ++mt) {
    // output adjoint (fp32) -> hi/lo A fragments
    uint32_t h3[KT3][4], l3[KT3][4];
    {
      float d3[2 * KT3][4];
#pragma unroll
      for (int nt = 0; nt < 2 * KT3; ++nt) {
        const int c = nt * 8 + 2 * q, r0 = mt * 16 + g, r1 = r0 + 8;
        d3[nt][0] = c < no ? ubar(c, r0) : 0.f;
        d3[nt][1] = c + 1 < no ? ubar(c + 1, r0) : 0.f;
        d3[nt][2] = c < no ? ubar(c, r1) : 0.f;
        d3[nt][3] = c + 1 < no ? ubar(c + 1, r1) : 0.f;
      }
      split_to_a<2 * KT3>(d3, h3, l3);
    }
    float s[NT0][4];
    zero_acc<NT0>(s);
#pragma unroll 1
    for (int c1 = 0; c1 < H1 / C1; ++c1) {
      float d1[NT1][4];
      zero_acc<NT1>(d1);
#pragma unroll 1
      for (int c2 = 0; c2 < H2 / C; ++c2) {
        float d2[NTC][4];
        zero_acc<NTC>(d2);
        mma_acc_split<KT3, NTC>(h3, l3, W3t, KT3 * 16, c2 * C, 0, d2);
        relu_mask<NTC>(d2, mask, 2, mt, c2 * C);
        if (c1 == 0) store_c<NTC>(d2, mt, c2 * C, H2, [&](int f, int r, float v) { del(2, f, r, v); });
        uint32_t h2[NTC / 2][4], l2[NTC / 2][4];
        split_to_a<NTC>(d2, h2, l2);
        mma_acc_split<NTC / 2, NT1>(h2, l2, W2t, H2, c1 * C1, c2 * C, d1);
      }
      relu_mask<NT1>(d1, mask, 1, mt, c1 * C1);
      store_c<NT1>(d1, mt, c1 * C1, H1, [&](int f, int r, float v) { del(1, f, r, v); });
      uint32_t h1[NT1 / 2][4], l1[NT1 / 2][4];
      split_to_a<NT1>(d1, h1, l1);
      mma_acc_split<NT1 / 2, NT0>(h1, l1, W1t, H1, 0, c1 * C1, s);
    }
    store_c<NT0>(s, mt, 0, k0, sbar);
  }
}
