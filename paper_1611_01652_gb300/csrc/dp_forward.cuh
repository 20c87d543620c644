// Forward step of the rigid-body engine, one lane per instance (arXiv 1611.01652, section 2.1):
// controller (Eq. g) -> servo targets -> gravity and gyroscopic impulses -> branchless sphere
// contact detection -> constraint rows -> fixed-iteration projected Gauss-Seidel -> semi-implicit
// Euler with the Eq. 1 renormalisation (read as R <- (3R - R R^T R)/2) -> loss term (Eq. L).
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "dp_device.cuh"
#include "dp_mma.cuh"

#define FULLMASK 0xffffffffu

// Tag of the run-time topology path (compile-time topologies are in dp_static.cuh).
struct DynTopo {
  static constexpr int id = 0;
};

// Views of one lane's data. RV is the constraint-row view: shared memory (SL) when the rows of
// 32 instances fit next to the rest of the warp's working set, else global memory (GL).
template <class RV>
struct LaneT {
  SL S;        // this warp's shared-memory block, offset to the lane
  GC P;        // parameters [field][Bp]
  RV rows;     // constraint rows, slot s at rows[s * RF_N + f]
  int i;       // instance index
};

template <class XV>
__device__ __forceinline__ float3 body_v(const XV& X, int b) { return b >= 0 ? X.v3(18 * b + 12) : f3(0.f, 0.f, 0.f); }
template <class XV>
__device__ __forceinline__ float3 body_w(const XV& X, int b) { return b >= 0 ? X.v3(18 * b + 15) : f3(0.f, 0.f, 0.f); }
template <class XV>
__device__ __forceinline__ float3 body_p(const XV& X, int b) { return b >= 0 ? X.v3(18 * b) : f3(0.f, 0.f, 0.f); }
template <class XV>
__device__ __forceinline__ M3 body_R(const XV& X, int b) { return b >= 0 ? loadRv(X, 18 * b) : eye3(); }

// Hinge axis (world), angle about it between the two reference vectors, and its rate.
// (jmask: the joints to process, bit j; the multi-warp kernels split them between warps)
template <class RV, class XV>
__device__ void hinge_kinematics(const DevTopo& T, const LaneT<RV>& L, const XV& X, uint32_t jmask = 0xffffffffu) {
  const SL& S = L.S;
  for (int j = 0; j < T.nj; ++j) {
    if (!((jmask >> j) & 1u)) continue;
    int a = T.ja[j], b = T.jb[j];
    M3 Ra = body_R(X, a);
    float3 ua = mv(Ra, L.P.v3(T.o_axis + 6 * j));
    S.s3(T.sm_ua + 3 * j, ua);
    if (T.jtype[j] == 1) {
      M3 Rb = loadRv(X, 18 * b);
      float3 wa = mv(Ra, L.P.v3(T.o_ref + 6 * j));
      float3 wb = mv(Rb, L.P.v3(T.o_ref + 6 * j + 3));
      float y = dot3(cross3(wa, wb), ua), x = dot3(wa, wb);
      S[T.sm_th + j] = atan2f(y, x);
      S[T.sm_thd + j] = dot3(ua, body_w(X, b) - body_w(X, a));
    } else {
      S[T.sm_th + j] = 0.f;
      S[T.sm_thd + j] = 0.f;
    }
  }
}

// Loss point q = p_b + R_b c.
template <class RV>
__device__ __forceinline__ float3 loss_point(const DevTopo& T, const LaneT<RV>& L, const SL& X) {
  int b = T.loss_body;
  return X.v3(18 * b) + mv(loadR(X, 18 * b), L.P.v3(T.o_loss_point));
}
template <class RV>
__device__ __forceinline__ float loss_value(const DevTopo& T, const LaneT<RV>& L, const SL& X) {
  float3 q = loss_point(T, L, X);
  float3 y = L.P.v3(T.o_loss_target);
  float3 d = q - y;
  switch (T.loss_kind) {
    case 0: return dot3(d, d);
    case 1: return sqrtf(dot3(d, d));
    default: return dot3(y, q);
  }
}
// Weight of l(x_{t_next}) in Eq. L for an instance of horizon h: the final state, or the mean
// over the states 1..h.
__device__ __forceinline__ float loss_weight(const DevTopo& T, int t_next, int h) {
  if (T.loss_mode == 1) return t_next <= h ? 1.f / (float)h : 0.f;
  return t_next == h ? 1.f : 0.f;
}
// Largest horizon among the warp's instances.
__device__ __forceinline__ int warp_horizon(const DevPtrs& D, int i) {
  int h = D.hz[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
  return h;
}

__device__ __forceinline__ float qz(const DevTopo& T, float x) { return T.ctrl_round ? bf16r(x) : x; }

// Controller input vector s(x^t), rounded to bfloat16 (unless the fp32 controller mode is
// selected), into act0 (padded with zeros).
template <class RV, class AV>
__device__ void controller_features(const DevTopo& T, const LaneT<RV>& L, const SL& X, int t, const AV& act0) {
  const SL& S = L.S;
  int k = 0;
  if (T.features & 1)
    for (int m = 0; m < T.n_motors; ++m) act0[k++] = qz(T, S[T.sm_th + T.motor_joint[m]]);
  if (T.features & 2)
    for (int m = 0; m < T.n_motors; ++m) act0[k++] = qz(T, S[T.sm_thd + T.motor_joint[m]]);
  if (T.features & 4) {
    double ph = 2.0 * 3.14159265358979323846 * (double)T.clock_hz * ((double)t * (double)T.dt);
    act0[k++] = qz(T, (float)sin(ph));
    act0[k++] = qz(T, (float)cos(ph));
  }
  if (T.features & 8) {
    int b = T.imu_body;
    M3 R = loadR(X, 18 * b);
    float3 g = mtv(R, f3(0.f, 0.f, -1.f));
    float3 wl = mtv(R, X.v3(18 * b + 15));
    act0[k++] = qz(T, g.x); act0[k++] = qz(T, g.y); act0[k++] = qz(T, g.z);
    act0[k++] = qz(T, wl.x); act0[k++] = qz(T, wl.y); act0[k++] = qz(T, wl.z);
  }
  if (T.features & 16) {
    float3 d = loss_point(T, L, X) - L.P.v3(T.o_loss_target);
    act0[k++] = qz(T, d.x); act0[k++] = qz(T, d.y); act0[k++] = qz(T, d.z);
  }
  for (; k < T.widths[0]; ++k) act0[k] = 0.f;
}

// One dense layer on this lane: out[o] = b[o] + sum_i W[o][i] in[i], weights from the
// [in][out_pad] copy (8 outputs per pass, broadcast float4 loads).
template <class AVI, class AVO>
__device__ void dense_fwd(const float* __restrict__ Wt, const float* __restrict__ bias, int ni, int no, const AVI& in,
                          const AVO& out, bool hidden, bool accumulate, bool round) {
  const int nop = (no + 7) & ~7;
  for (int o0 = 0; o0 < no; o0 += 8) {
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = (o0 + k < no) ? __ldg(bias + o0 + k) : 0.f;
    const float* w = Wt + o0;
    for (int ii = 0; ii < ni; ++ii) {
      float av = in[ii];
      float4 w0 = __ldg(reinterpret_cast<const float4*>(w + (size_t)ii * nop));
      float4 w1 = __ldg(reinterpret_cast<const float4*>(w + (size_t)ii * nop + 4));
      acc[0] = fmaf(w0.x, av, acc[0]); acc[1] = fmaf(w0.y, av, acc[1]);
      acc[2] = fmaf(w0.z, av, acc[2]); acc[3] = fmaf(w0.w, av, acc[3]);
      acc[4] = fmaf(w1.x, av, acc[4]); acc[5] = fmaf(w1.y, av, acc[5]);
      acc[6] = fmaf(w1.z, av, acc[6]); acc[7] = fmaf(w1.w, av, acc[7]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (o0 + k < no) {
        float z = accumulate ? out[o0 + k] + acc[k] : acc[k];
        out[o0 + k] = hidden ? (round ? bf16r(fmaxf(z, 0.f)) : fmaxf(z, 0.f)) : z;
      }
    }
  }
}

// Controller forward: act[0] already holds the features; act[n_layers] gets the output u.
template <class AV>
__device__ void controller_forward(const DevTopo& T, const DevPtrs& D, const AV* act) {
  for (int l = 0; l < T.n_layers; ++l) {
    const int ni = T.widths[l], no = T.widths[l + 1];
    const float* Wt = D.Wt + T.w_off[l];
    const float* b = D.bias + T.w_off[l];
    dense_fwd(Wt, b, ni, no, act[l], act[l + 1], l + 1 < T.n_layers, false, T.ctrl_round != 0);
  }
  if (T.skip) {
    const int l = T.n_layers;
    dense_fwd(D.Wt + T.w_off[l], D.bias + T.w_off[l], T.widths[0], T.widths[l], act[0], act[l], false, true, false);
  }
}

// Hidden widths of the tensor-core controller a kernel is built for: a compiled topology carries
// one width (Q::CTRL_H); the run-time topology every supported width.
template <class Q, class F>
__device__ __forceinline__ void ctrl_tc_dispatch(const DevTopo& T, F&& f) {
  if constexpr (Q::id != 0) {
    f(std::integral_constant<int, Q::CTRL_H>{});
  } else {
    if (T.widths[1] == 64) f(std::integral_constant<int, 64>{});
    else if (T.widths[1] == 128) f(std::integral_constant<int, 128>{});
    else f(std::integral_constant<int, 256>{});
  }
}

// Controller forward on the tensor cores (a bfloat16 K0-H-H-NO network, K0 <= 32, NO <= 16, H in
// {64, 128, 256}): the warp's 32 instances are the rows of each product. act[0] holds the
// features, act[3] receives the outputs. Hidden activations go to the dump column when one is
// given, to act[1], act[2] when those are dump views (segment recompute), and nowhere otherwise.
template <int H, class AV>
__device__ __forceinline__ void ctrl_tc_forward(const DevTopo& T, const DevPtrs& D, const AV* act, float* dump_col,
                                                int mt0 = 0, int mt1 = 2) {
  const __nv_bfloat16* Wc = D.Wtc;
  const size_t N = (size_t)T.horizon * T.Bp;
  const int lane = threadIdx.x & 31;
  float* dbase = dump_col ? dump_col - lane : nullptr;
  const int d1 = T.dump_act[1], d2 = T.dump_act[2];
  const AV a0 = act[0], a1 = act[1], a2 = act[2], a3 = act[3];
  constexpr CtrlTCLayout Lw = ctrl_tc_layout(H, H);
  mlp3_forward<CTRL_TC_KP0, H, H, CTRL_TC_NOP>(
      T.widths[0], T.widths[3], [&](int f, int r) { return a0.lane_at(f, r); }, Wc + Lw.w1, D.bias + T.w_off[0],
      Wc + Lw.w2, D.bias + T.w_off[1], Wc + Lw.w3, D.bias + T.w_off[2],
      [&](int f, int r, float v) { a3.lane_at(f, r) = v; },
      [&](int l, int f, int r, float v) {
        if (dbase)
          dbase[(size_t)((l == 1 ? d1 : d2) + f) * N + r] = v;
        else if constexpr (!std::is_same<AV, SL>::value)
          (l == 1 ? a1 : a2).lane_at(f, r) = v;
      },
      mt0, mt1);
}
// The run-time topology's kernels (and the compiled ones with the 256-wide network) call the
// controller out of line, so that the register needs of the widest network do not fall on the
// whole persistent kernel.
template <int H, class AV>
__device__ __noinline__ void ctrl_tc_forward_call(const DevTopo& T, const DevPtrs& D, const AV* act, float* dump_col,
                                                  int mt0 = 0, int mt1 = 2) {
  ctrl_tc_forward<H, AV>(T, D, act, dump_col, mt0, mt1);
}
// Controller forward of a compiled topology's kernel (its one width), 16-row tiles mt0 .. mt1 - 1.
template <class Q, class AV>
__device__ __forceinline__ void ctrl_tc_forward_q(const DevTopo& T, const DevPtrs& D, const AV* act, float* dump_col,
                                                  int mt0 = 0, int mt1 = 2) {
  if constexpr (Q::CTRL_H <= 128)
    ctrl_tc_forward<Q::CTRL_H, AV>(T, D, act, dump_col, mt0, mt1);
  else
    ctrl_tc_forward_call<Q::CTRL_H, AV>(T, D, act, dump_col, mt0, mt1);
}
template <class Q, class AV>
__device__ void controller_forward_tc(const DevTopo& T, const DevPtrs& D, const AV* act, float* dump_col) {
  __syncwarp();
  if constexpr (Q::id != 0) {
    ctrl_tc_forward_q<Q, AV>(T, D, act, dump_col);
  } else {
    if (T.widths[1] == 64) ctrl_tc_forward_call<64, AV>(T, D, act, dump_col);
    else if (T.widths[1] == 128) ctrl_tc_forward_call<128, AV>(T, D, act, dump_col);
    else ctrl_tc_forward_call<256, AV>(T, D, act, dump_col);
  }
  __syncwarp();
}

// Servo targets w* = clamp(k (u - theta), -vmax, vmax).
template <class RV, class AV>
__device__ void servo_targets(const DevTopo& T, const LaneT<RV>& L, const AV& u, uint32_t jmask = 0xffffffffu) {
  const SL& S = L.S;
  for (int m = 0; m < T.n_motors; ++m) {
    int j = T.motor_joint[m];
    if (!((jmask >> j) & 1u)) continue;
    float k = L.P[T.o_motor + 3 * j], vmax = L.P[T.o_motor + 3 * j + 2];
    float um = (T.n_layers > 0 && m < T.widths[T.n_layers]) ? u[m] : 0.f;
    float x = k * (um - S[T.sm_th + j]);
    float br = x < -vmax ? 1.f : (x > vmax ? 2.f : 0.f);
    S[T.sm_wst + j] = br == 1.f ? -vmax : (br == 2.f ? vmax : x);
    S[T.sm_wbr + j] = br;
  }
}

// Gravity and the explicit gyroscopic term; world inverse inertia and inverse mass (bmask: the
// bodies to process, bit b).
template <class RV>
__device__ void external_impulses(const DevTopo& T, const LaneT<RV>& L, const SL& X, uint32_t bmask = 0xffffffffu) {
  const SL& S = L.S;
  const float h = T.dt;
  const float3 g = f3(T.gravity[0], T.gravity[1], T.gravity[2]);
  for (int b = 0; b < T.nb; ++b) {
    if (!((bmask >> b) & 1u)) continue;
    M3 R = loadR(X, 18 * b);
    float3 I = L.P.v3(T.o_inertia + 3 * b);
    float m = L.P[T.o_mass + b];
    float iw[6], ii[6];
    rot_diag6(R, I, iw);
    rot_diag6(R, f3(1.f / I.x, 1.f / I.y, 1.f / I.z), ii);
    float3 v = X.v3(18 * b + 12) + h * g;
    float3 w = X.v3(18 * b + 15);
    float3 gy = -cross3(w, symv(iw, w));
    w += h * symv(ii, gy);
    X.s3(18 * b + 12, v);
    X.s3(18 * b + 15, w);
    S[T.sm_invm + b] = 1.f / m;
#pragma unroll
    for (int k = 0; k < 6; ++k) S[T.sm_iinv + 6 * b + k] = ii[k];
  }
}

// World inverse inertia and inverse mass of every body at state X (no state change; bmask:
// the bodies to process, bit b).
template <class RV, class XV>
__device__ void inverse_inertia(const DevTopo& T, const LaneT<RV>& L, const XV& X, uint32_t bmask = 0xffffffffu) {
  const SL& S = L.S;
  for (int b = 0; b < T.nb; ++b) {
    if (!((bmask >> b) & 1u)) continue;
    M3 R = loadRv(X, 18 * b);
    float3 I = L.P.v3(T.o_inertia + 3 * b);
    float ii[6];
    rot_diag6(R, f3(1.f / I.x, 1.f / I.y, 1.f / I.z), ii);
    S[T.sm_invm + b] = 1.f / L.P[T.o_mass + b];
#pragma unroll
    for (int k = 0; k < 6; ++k) S[T.sm_iinv + 6 * b + k] = ii[k];
  }
}

__device__ __forceinline__ float min0f(float x) { return x < 0.f ? x : 0.f; }

// Geometry of one contact/joint row; shared by assembly and its reverse mode.
struct RowGeo {
  float3 lin, angA, angB;
  float bias, lo, hi;
  bool active;
};

// Assemble constraint slots s0, s0 + sstep, ... of this instance into rows (every slot by
// default; each slot's row depends on the state alone, so the slots may be split over warps).
template <class RV>
__device__ void assemble_rows(const DevTopo& T, const LaneT<RV>& L, const SL& X, uint8_t* active_out, int s0 = 0,
                              int sstep = 1) {
  const SL& S = L.S;
  const float h = T.dt;
  const float bh = T.beta / h;
  const float INF = __int_as_float(0x7f800000);
  const float3 ez = f3(0.f, 0.f, 1.f);
  for (int s = s0; s < T.nslots; s += sstep) {
    const int kind = T.skind[s], idx = T.sidx[s], sub = T.ssub[s], a = T.sa[s], b = T.sb[s];
    float3 lin = f3(0.f, 0.f, 0.f), angA = lin, angB = lin;
    float bias = 0.f, bnd = 0.f;
    bool active = true;
    switch (kind) {
      case RK_JLIN: {
        float3 ra = a >= 0 ? mv(loadR(X, 18 * a), L.P.v3(T.o_anchor + 6 * idx)) : L.P.v3(T.o_anchor + 6 * idx);
        float3 rb = mv(loadR(X, 18 * b), L.P.v3(T.o_anchor + 6 * idx + 3));
        float3 C = (body_p(X, a) + ra) - (X.v3(18 * b) + rb);
        float3 e = f3(sub == 0 ? 1.f : 0.f, sub == 1 ? 1.f : 0.f, sub == 2 ? 1.f : 0.f);
        lin = e;
        angA = a >= 0 ? cross3(ra, e) : f3(0.f, 0.f, 0.f);
        angB = -cross3(rb, e);
        bias = bh * (sub == 0 ? C.x : (sub == 1 ? C.y : C.z));
        break;
      }
      case RK_JANG: {
        float3 t1, t2;
        onb3(L.P.v3(T.o_axis + 6 * idx), t1, t2);
        float3 t = mv(body_R(X, a), sub == 0 ? t1 : t2);
        float3 ub = mv(loadR(X, 18 * b), L.P.v3(T.o_axis + 6 * idx + 3));
        float3 ua = S.v3(T.sm_ua + 3 * idx);
        angA = a >= 0 ? t : f3(0.f, 0.f, 0.f);
        angB = -t;
        bias = bh * dot3(t, cross3(ub, ua));
        break;
      }
      case RK_LIMIT: {
        float th = S[T.sm_th + idx];
        float lo_j = L.P[T.o_limit + 2 * idx], hi_j = L.P[T.o_limit + 2 * idx + 1];
        float3 ua = S.v3(T.sm_ua + 3 * idx);
        if (th <= lo_j) {
          angA = a >= 0 ? -ua : f3(0.f, 0.f, 0.f); angB = ua; bias = bh * (th - lo_j);
        } else if (th >= hi_j) {
          angA = a >= 0 ? ua : f3(0.f, 0.f, 0.f); angB = -ua; bias = bh * (hi_j - th);
        } else {
          active = false;
        }
        break;
      }
      case RK_MOTOR: {
        float3 ua = S.v3(T.sm_ua + 3 * idx);
        angA = a >= 0 ? -ua : f3(0.f, 0.f, 0.f);
        angB = ua;
        bias = -S[T.sm_wst + idx];
        bnd = L.P[T.o_motor + 3 * idx + 1] * h;
        break;
      }
      case RK_GN:
      case RK_GT: {
        float3 c = mv(loadR(X, 18 * a), L.P.v3(T.o_sph_off + 3 * idx));
        float rad = L.P[T.o_sph_rad + idx];
        float d = (X[18 * a + 2] + c.z) - rad - T.ground_z;
        active = d <= 0.f;
        float3 ra = c - rad * ez;
        if (kind == RK_GN) {
          lin = ez;
          angA = cross3(ra, ez);
          float vn = dot3(lin, X.v3(18 * a + 12)) + dot3(angA, X.v3(18 * a + 15));
          bias = bh * min0f(d + T.slop) + L.P[T.o_sph_e + idx] * min0f(vn);
        } else {
          lin = sub == 0 ? f3(1.f, 0.f, 0.f) : f3(0.f, 1.f, 0.f);  // basis of +z
          angA = cross3(ra, lin);
          bnd = L.P[T.o_sph_mu + idx];
        }
        break;
      }
      case RK_PN:
      case RK_PT: {
        const int k = T.pk[idx], l = T.pl[idx];
        float3 ck = mv(loadR(X, 18 * a), L.P.v3(T.o_sph_off + 3 * k));
        float3 cl = mv(loadR(X, 18 * b), L.P.v3(T.o_sph_off + 3 * l));
        float3 dl = (X.v3(18 * a) + ck) - (X.v3(18 * b) + cl);
        float dist = sqrtf(dot3(dl, dl));
        float3 n = dist > 1e-9f ? (1.f / dist) * dl : ez;
        float rk = L.P[T.o_sph_rad + k], rl = L.P[T.o_sph_rad + l];
        float d = dist - rk - rl;
        active = d <= 0.f;
        float3 ra = ck - rk * n, rb = cl + rl * n;
        if (kind == RK_PN) {
          lin = n;
          angA = cross3(ra, n);
          angB = -cross3(rb, n);
          float vn = dot3(n, X.v3(18 * a + 12) - X.v3(18 * b + 12)) + dot3(angA, X.v3(18 * a + 15)) +
                     dot3(angB, X.v3(18 * b + 15));
          float ek = L.P[T.o_sph_e + k], el = L.P[T.o_sph_e + l];
          float e = ek >= el ? ek : el;
          bias = bh * min0f(d + T.slop) + e * min0f(vn);
        } else {
          float3 t1, t2;
          onb3(n, t1, t2);
          lin = sub == 0 ? t1 : t2;
          angA = cross3(ra, lin);
          angB = -cross3(rb, lin);
          bnd = sqrtf(L.P[T.o_sph_mu + k] * L.P[T.o_sph_mu + l]);
        }
        break;
      }
    }
    float3 IA = f3(0.f, 0.f, 0.f), IB = IA;
    float K = 0.f;
    if (a >= 0) {
      float ia[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ia[q] = S[T.sm_iinv + 6 * a + q];
      IA = symv(ia, angA);
      K += S[T.sm_invm + a] * dot3(lin, lin) + dot3(angA, IA);
    }
    if (b >= 0) {
      float ib[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ib[q] = S[T.sm_iinv + 6 * b + q];
      IB = symv(ib, angB);
      K += S[T.sm_invm + b] * dot3(lin, lin) + dot3(angB, IB);
    }
    const RV R = L.rows.at(s * RF_N);
    R.s3(RF_LIN, lin);
    R.s3(RF_ANGA, angA);
    R.s3(RF_ANGB, angB);
    R.s3(RF_IA, IA);
    R.s3(RF_IB, IB);
    R[RF_MEFF] = active ? 1.f / (K + T.gamma) : 0.f;
    R[RF_BIAS] = active ? bias : 0.f;
    R[RF_BND] = bnd;
    if (active_out) active_out[s] = active ? 1 : 0;
  }
}

// Projected Gauss-Seidel, cold start, T.iters sweeps in the canonical order. With TAPE the
// impulses and clamp branches of every sweep and the velocities after every sweep are kept.
template <bool TAPE, class RV>
__device__ void pgs_solve(const DevTopo& T, const LaneT<RV>& L, const SL& X, const TapeStep& tp) {
  const SL& S = L.S;
  const int Bp = T.Bp;
  if (!T.ws)
    for (int s = 0; s < T.nslots; ++s) S[T.sm_lam + s] = 0.f;
  for (int it = 0; it < T.iters; ++it) {
    for (int oi = 0; oi < T.nslots; ++oi) {
      const int s = T.order[oi];
      const RV R = L.rows.at(s * RF_N);
      const float meff = R[RF_MEFF];
      if (!__any_sync(FULLMASK, meff != 0.f)) continue;  // the row is inactive on every lane
      const int kind = T.skind[s], a = T.sa[s], b = T.sb[s];
      const float3 lin = R.v3(RF_LIN);
      const float3 angA = R.v3(RF_ANGA), angB = R.v3(RF_ANGB);
      const float bias = R[RF_BIAS];
      const float lam = S[T.sm_lam + s];
      float lo, hi;
      if (kind == RK_GT || kind == RK_PT) {
        hi = R[RF_BND] * S[T.sm_lam + T.snormal[s]];
        lo = -hi;
      } else if (kind == RK_MOTOR) {
        hi = R[RF_BND];
        lo = -hi;
      } else if (kind == RK_JLIN || kind == RK_JANG) {
        lo = -__int_as_float(0x7f800000);
        hi = __int_as_float(0x7f800000);
      } else {
        lo = 0.f;
        hi = __int_as_float(0x7f800000);
      }
      float Jv = 0.f;
      float3 va, wa, vb, wb;
      const SL Xa = X.at(18 * a + 12), Xb = X.at(18 * b + 12);
      if (a >= 0) { va = Xa.v3(0); wa = Xa.v3(3); Jv += dot3(lin, va) + dot3(angA, wa); }
      if (b >= 0) { vb = Xb.v3(0); wb = Xb.v3(3); Jv += dot3(angB, wb) - dot3(lin, vb); }
      const float pre = lam - meff * (Jv + bias + T.gamma * lam);
      const int br = pre < lo ? 1 : (pre > hi ? 2 : 0);
      const float ln = br == 1 ? lo : (br == 2 ? hi : pre);
      const float dl = ln - lam;
      S[T.sm_lam + s] = ln;
      if (a >= 0) {
        Xa.s3(0, va + (dl * S[T.sm_invm + a]) * lin);
        Xa.s3(3, wa + dl * R.v3(RF_IA));
      }
      if (b >= 0) {
        Xb.s3(0, vb - (dl * S[T.sm_invm + b]) * lin);
        Xb.s3(3, wb + dl * R.v3(RF_IB));
      }
      if (TAPE) {
        const int o = (it * T.nslots + s) * 32;
        tp.lam[o] = ln;
        tp.br[o] = (uint8_t)br;
      }
    }
    if (TAPE) {
      float* vi = tp.viter + it * T.nb * 6 * 32;
      for (int b = 0; b < T.nb; ++b)
#pragma unroll
        for (int k = 0; k < 6; ++k) vi[(6 * b + k) * 32] = X[18 * b + 12 + k];
    }
  }
}

// Semi-implicit Euler on positions with the new velocities, then the Eq. 1 renormalisation.
__device__ inline void integrate(const DevTopo& T, const SL& X, uint32_t bmask = 0xffffffffu) {
  const float h = T.dt;
  for (int b = 0; b < T.nb; ++b) {
    if (!((bmask >> b) & 1u)) continue;
    float3 p = X.v3(18 * b), v = X.v3(18 * b + 12), w = X.v3(18 * b + 15);
    M3 R = loadR(X, 18 * b), A;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.m[j] = R.m[j] + h * (-w.z * R.m[3 + j] + w.y * R.m[6 + j]);
      A.m[3 + j] = R.m[3 + j] + h * (w.z * R.m[j] - w.x * R.m[6 + j]);
      A.m[6 + j] = R.m[6 + j] + h * (-w.y * R.m[j] + w.x * R.m[3 + j]);
    }
    M3 AAA = mm(A, mm(mT(A), A));
    X.s3(18 * b, p + h * v);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[18 * b + 3 + k] = 0.5f * (3.f * A.m[k] - AAA.m[k]);
  }
}

// ------------------------------------------------------------------------------ warm start
// Learned warm start. The rows are taken in groups of three (DevTopo.wsg_*): the linear rows of
// a joint, the angular rows of a hinge with its motor row, the normal and friction rows of a
// contact. Each group gets 16 features from its assembled rows, the pre-solve velocities and the
// robot's mass distribution; the 16-64-64-3 bfloat16 network (tensor cores, the warp's 32
// instances as rows) gives a velocity-scale correction y per row, and the start alpha
// lambda_prev + m_eff y is projected on the rows' bounds (normal >= 0, |friction| <= mu normal,
// |motor| <= tau_max h) and applied in slot order before the first sweep. The same features
// feed the harvest of training rows.
template <class RV>
__device__ __forceinline__ float row_jv(const DevTopo& T, const RV& R, const SL& X, int a, int b) {
  float Jv = 0.f;
  const float3 lin = R.v3(RF_LIN);
  if (a >= 0) Jv += dot3(lin, X.v3(18 * a + 12)) + dot3(R.v3(RF_ANGA), X.v3(18 * a + 15));
  if (b >= 0) Jv += dot3(R.v3(RF_ANGB), X.v3(18 * b + 15)) - dot3(lin, X.v3(18 * b + 12));
  return Jv;
}

// Applies impulse dl of row R (slot bodies a, b) to the velocities in X.
template <class RV>
__device__ __forceinline__ void row_apply(const DevTopo& T, const SL& S, const RV& R, const SL& X, int a, int b, float dl,
                                          uint32_t bmask = 0xffffffffu) {
  const float3 lin = R.v3(RF_LIN);
  if (a >= 0 && ((bmask >> a) & 1u)) {
    X.s3(18 * a + 12, X.v3(18 * a + 12) + (dl * S[T.sm_invm + a]) * lin);
    X.s3(18 * a + 15, X.v3(18 * a + 15) + dl * R.v3(RF_IA));
  }
  if (b >= 0 && ((bmask >> b) & 1u)) {
    X.s3(18 * b + 12, X.v3(18 * b + 12) - (dl * S[T.sm_invm + b]) * lin);
    X.s3(18 * b + 15, X.v3(18 * b + 15) + dl * R.v3(RF_IB));
  }
}

// Projection of row group g's start z onto its rows' bounds, into S[sm_lam]: normal >= 0,
// |friction| <= mu lambda0_n, |motor| <= tau_max h, inactive rows 0.
template <class RV>
__device__ __forceinline__ void ws_project(const DevTopo& T, const LaneT<RV>& L, int g, const float (&z)[3]) {
  const SL& S = L.S;
  const int type = T.wsg_type[g];
  const int s0 = T.wsg_slot[g][0], s1 = T.wsg_slot[g][1], s2 = T.wsg_slot[g][2];
  const bool active = L.rows[s0 * RF_N + RF_MEFF] != 0.f;
  if (type == WSG_GROUND || type == WSG_PAIR) {
    float l0[3] = {0.f, 0.f, 0.f};
    if (active) {
      l0[0] = fmaxf(z[0], 0.f);
      const float hi = L.rows[s1 * RF_N + RF_BND] * l0[0];
      l0[1] = fminf(fmaxf(z[1], -hi), hi);
      l0[2] = fminf(fmaxf(z[2], -hi), hi);
    }
    S[T.sm_lam + s0] = l0[0];
    S[T.sm_lam + s1] = l0[1];
    S[T.sm_lam + s2] = l0[2];
  } else {
    for (int k = 0; k < 3; ++k) {
      const int s = T.wsg_slot[g][k];
      if (s < 0) continue;
      float y = L.rows[s * RF_N + RF_MEFF] != 0.f ? z[k] : 0.f;
      if (T.skind[s] == RK_MOTOR) {
        const float hi = L.rows[s * RF_N + RF_BND];
        y = fminf(fmaxf(y, -hi), hi);
      }
      S[T.sm_lam + s] = y;
    }
  }
}

// Features, inference, projection and application (ws), harvest row reservation (harvest).
// On entry S[sm_lam] holds the impulses the previous step ended with (lambda_prev); on exit the
// initial impulses alpha lambda_prev + network output, projected (warm start), or the same
// lambda_prev (cold start: the solver zeroes them).
template <bool TAPE, class RV>
__device__ void warm_start(const DevTopo& T, const DevPtrs& D, const LaneT<RV>& L, const SL& X, const TapeStep& tp) {
  const SL& S = L.S;
  const bool harvest = D.harvest != nullptr;
  // the features are needed by a nonzero network and by the harvest; with an identically zero
  // network the start is alpha * (previous impulses) + m_eff * 0, computed without them
  const bool feat = harvest || (T.ws && T.ws_net);
  float mtot = 0.f;
  float3 pc = f3(0.f, 0.f, 0.f);
  int nact = 0;
  float share = 0.f;
  if (feat) {
    for (int b = 0; b < T.nb; ++b) {
      const float m = L.P[T.o_mass + b];
      mtot += m;
      pc += m * X.v3(18 * b);
    }
    pc = (1.f / mtot) * pc;
    for (int s = 0; s < T.nslots; ++s)
      if ((T.skind[s] == RK_GN || T.skind[s] == RK_PN) && L.rows[s * RF_N + RF_MEFF] != 0.f) ++nact;
    const float gn = sqrtf(T.gravity[0] * T.gravity[0] + T.gravity[1] * T.gravity[1] + T.gravity[2] * T.gravity[2]);
    share = mtot * gn * T.dt / (float)max(1, nact);
  }
  const SL F = S.at(T.sm_ws), Y = S.at(T.sm_ws + 16), H = S.at(T.sm_ws + 19);
  const int lane = threadIdx.x & 31;
  for (int g = 0; g < T.n_wsg; ++g) {
    const int type = T.wsg_type[g];
    const int s0 = T.wsg_slot[g][0], s1 = T.wsg_slot[g][1], s2 = T.wsg_slot[g][2];
    const bool contact = type == WSG_GROUND || type == WSG_PAIR;
    float lp[3];  // impulses the group's rows ended the previous step with
    for (int k = 0; k < 3; ++k) {
      const int s = T.wsg_slot[g][k];
      lp[k] = s >= 0 ? S[T.sm_lam + s] : 0.f;
    }
    if (feat) {
    float3 q;  // the group's point: contact point on body a, or the joint's anchor on its child
    if (type == WSG_GROUND) {
      const int qi = T.sidx[s0], a = T.sa[s0];
      q = X.v3(18 * a) + mv(loadR(X, 18 * a), L.P.v3(T.o_sph_off + 3 * qi)) - L.P[T.o_sph_rad + qi] * f3(0.f, 0.f, 1.f);
    } else if (type == WSG_PAIR) {
      const int k = T.pk[T.sidx[s0]], a = T.sa[s0];
      q = X.v3(18 * a) + mv(loadR(X, 18 * a), L.P.v3(T.o_sph_off + 3 * k)) -
          L.P[T.o_sph_rad + k] * L.rows.at(s0 * RF_N).v3(RF_LIN);
    } else {
      const int j = T.sidx[s0], b = T.sb[s0];
      q = X.v3(18 * b) + mv(loadR(X, 18 * b), L.P.v3(T.o_anchor + 6 * j + 3));
    }
    for (int k = 0; k < 3; ++k) {
      const int s = T.wsg_slot[g][k];
      const RV R = L.rows.at((s >= 0 ? s : 0) * RF_N);
      const bool on = s >= 0 && R[RF_MEFF] != 0.f;  // rows of inactive slots contribute zeros
      F[k] = on ? row_jv(T, R, X, T.sa[s], T.sb[s]) : 0.f;
      F[3 + k] = on ? R[RF_BIAS] : 0.f;
      F[6 + k] = on ? R[RF_MEFF] : 0.f;
    }
    F[9] = contact ? L.rows[s1 * RF_N + RF_BND] : (type == WSG_HINGE && s2 >= 0 ? L.rows[s2 * RF_N + RF_BND] : 0.f);
    F[10] = q.x - pc.x;
    F[11] = q.y - pc.y;
    F[12] = (float)nact;
    F[13] = share;
    F[14] = q.z - T.ground_z;
    F[15] = (float)type;
    }
    const bool active = L.rows[s0 * RF_N + RF_MEFF] != 0.f;
    if (harvest) {  // padded lanes (copies of the last instance) harvest nothing
      const unsigned m = __ballot_sync(FULLMASK, active && L.i < T.B);
      unsigned long long base = 0;
      if (lane == 0 && m) base = atomicAdd(D.harvest_count, (unsigned long long)__popc(m));
      base = __shfl_sync(FULLMASK, base, 0);
      const long long id = (m >> lane) & 1u ? (long long)(base + __popc(m & ((1u << lane) - 1u))) : -1;
      const bool keep = id >= 0 && id < D.harvest_max;
      H[g] = __int_as_float(keep ? (int)id : -1);
      if (keep) {
        for (int k = 0; k < 16; ++k) D.harvest[id * 19 + k] = F[k];
        for (int k = 0; k < 3; ++k) D.harvest[id * 19 + 16 + k] = lp[k];  // replaced after the solve
      }
    }
    if (T.ws) {
      float z[3];
      if (T.ws_net) {
        __syncwarp();
        mlp3_forward<WsTC::K0, WsTC::H1, WsTC::H2, WsTC::NO>(
            WsTC::K0, WsTC::NO,
            [&](int f, int r) { return F.lane_at(f, r); }, D.ws_tc + WsTC::W1, D.ws_b + WsTC::B1, D.ws_tc + WsTC::W2,
            D.ws_b + WsTC::B2, D.ws_tc + WsTC::W3, D.ws_b + WsTC::B3,
            [&](int f, int r, float v) { Y.lane_at(f, r) = v; }, [](int, int, int, float) {});
        __syncwarp();
        for (int k = 0; k < 3; ++k) z[k] = T.ws_alpha * lp[k] + F[6 + k] * Y[k];
      } else {
        for (int k = 0; k < 3; ++k) z[k] = T.ws_alpha * lp[k];
      }
      ws_project(T, L, g, z);
      __syncwarp();
    }
  }
  if (T.ws) {
    for (int s = 0; s < T.nslots; ++s)
      if (T.skind[s] == RK_LIMIT) S[T.sm_lam + s] = 0.f;  // limits start cold
    for (int s = 0; s < T.nslots; ++s) {
      const float l0 = S[T.sm_lam + s];
      if (l0 != 0.f) row_apply(T, S, L.rows.at(s * RF_N), X, T.sa[s], T.sb[s], l0);
    }
    if (TAPE)
      for (int s = 0; s < T.nslots; ++s) tp.lam0[s * 32] = S[T.sm_lam + s];
  }
}

// Harvest: per reserved group, the network's ideal output: the impulses after the solve minus
// alpha times the previous ones (parked in the row's output slots before the solve), divided by
// the row's effective mass (zero for inactive rows).
template <class RV>
__device__ void harvest_finish(const DevTopo& T, const DevPtrs& D, const LaneT<RV>& L) {
  const SL& S = L.S;
  const SL H = S.at(T.sm_ws + 19);
  for (int g = 0; g < T.n_wsg; ++g) {
    const int id = __float_as_int(H[g]);
    if (id < 0) continue;
    float* row = D.harvest + (long long)id * 19;
    for (int k = 0; k < 3; ++k) {
      const int s = T.wsg_slot[g][k];
      const float me = row[6 + k];
      row[16 + k] = me != 0.f ? ((s >= 0 ? S[T.sm_lam + s] : 0.f) - T.ws_alpha * row[16 + k]) / me : 0.f;
    }
  }
}

// RMS complementarity residual of the solve over the active rows, with w = J v + bias + gamma
// lambda: bilateral |w|; one-sided |min(lambda, w)|; boxed |lambda - clamp(lambda - w, lo, hi)|.
template <class RV>
__device__ float solve_residual(const DevTopo& T, const LaneT<RV>& L, const SL& X) {
  const SL& S = L.S;
  float ss = 0.f;
  int na = 0;
  for (int s = 0; s < T.nslots; ++s) {
    const RV R = L.rows.at(s * RF_N);
    if (R[RF_MEFF] == 0.f) continue;
    const int kind = T.skind[s];
    const float l = S[T.sm_lam + s];
    const float w = row_jv(T, R, X, T.sa[s], T.sb[s]) + R[RF_BIAS] + T.gamma * l;
    float e;
    if (kind == RK_JLIN || kind == RK_JANG) {
      e = w;
    } else if (kind == RK_LIMIT || kind == RK_GN || kind == RK_PN) {
      e = fminf(l, w);
    } else {
      const float hi = (kind == RK_MOTOR) ? R[RF_BND] : R[RF_BND] * S[T.sm_lam + T.snormal[s]];
      e = l - fminf(fmaxf(l - w, -hi), hi);
    }
    ss += e * e;
    ++na;
  }
  return na ? sqrtf(ss / (float)na) : 0.f;
}

// One full step x_t -> x_{t+1} in place on X. Returns the loss term of x_{t+1}.
template <class Q, bool TAPE, class RV>
__device__ void pgs_solve_static(const DevTopo& T, const LaneT<RV>& L, const SL& X, const TapeStep& tp);

// One full step x_t -> x_{t+1} in place on X. With TAPE the step's solver tape is written to
// slot `ts` of the tape (rows are copied there when they are assembled on chip) and, when
// `dump_col` is given, the controller activations are stored in the dump column.
template <bool TAPE, class Q = DynTopo, class RV, class AV>
__device__ float step_forward(const DevTopo& T, const DevPtrs& D, const LaneT<RV>& L, const SL& X, const AV* act, int t,
                              uint8_t* active_out, int ts = 0, float* dump_col = nullptr) {
  hinge_kinematics(T, L, X);
  if (T.ext_ctrl) {
    // wide controller: its output for this step was computed between launches
    const float* ue = D.u_ext + ((size_t)t * T.Bp + L.i) * T.ext_nop;
    for (int m = 0; m < T.widths[T.n_layers]; ++m) act[T.n_layers][m] = ue[m];
    servo_targets(T, L, act[T.n_layers]);
  } else if (T.n_layers > 0) {
    controller_features(T, L, X, t, act[0]);
    if (T.n_rec) {  // recurrent state h^t: the last inputs (a bfloat16 storage point like the sensors)
      const int base = T.widths[0] - T.n_rec;
      for (int k = 0; k < T.n_rec; ++k) act[0][base + k] = qz(T, L.S[T.sm_h + k]);
    }
    if (T.mlp_tc)
      controller_forward_tc<Q>(T, D, act, dump_col);
    else
      controller_forward(T, D, act);
    if (T.n_rec) {  // h^{t+1} = tanh of the last outputs
      const int base = T.widths[T.n_layers] - T.n_rec;
      for (int k = 0; k < T.n_rec; ++k) L.S[T.sm_h + k] = tanhf(act[T.n_layers][base + k]);
    }
    if (D.u_noise) {  // perturbed controller output (harvest of training rows)
      const float* nz = D.u_noise + ((size_t)t * T.B + min(L.i, T.B - 1)) * T.n_motors;  // [T][B][n_motors]
      for (int m = 0; m < T.n_motors && m < T.widths[T.n_layers]; ++m) act[T.n_layers][m] += nz[m];
    }
    if (dump_col) {
      const size_t N = (size_t)T.horizon * T.Bp;
      for (int l = 0; l <= T.n_layers; ++l) {
        if (T.mlp_tc && l > 0 && l < T.n_layers) continue;  // hidden layers went straight to the dump
        for (int k = 0; k < T.widths[l]; ++k) dump_col[(size_t)(T.dump_act[l] + k) * N] = act[l][k];
      }
    }
    servo_targets(T, L, act[T.n_layers]);
  } else {
    servo_targets(T, L, act[0]);
  }
  external_impulses(T, L, X);
  TapeStep tp;
  if (TAPE) {
    tp = tape_step(T, D, ts);
    for (int b = 0; b < T.nb; ++b)
#pragma unroll
      for (int k = 0; k < 6; ++k) tp.vminus[(6 * b + k) * 32] = X[18 * b + 12 + k];
  }
  assemble_rows(T, L, X, active_out);
  // the rows go to the tape, unless they were assembled in it (segment recompute)
  if constexpr (TAPE && !std::is_same<RV, GS>::value) {
    for (int f = 0; f < T.nslots * RF_N; ++f) tp.rows[f * 32] = L.rows[f];
  }
  if (T.ws || D.harvest) warm_start<TAPE>(T, D, L, X, tp);
  if constexpr (Q::id == 0)
    pgs_solve<TAPE>(T, L, X, tp);
  else
    pgs_solve_static<Q, TAPE>(T, L, X, tp);
  if (D.harvest) harvest_finish(T, D, L);
  if (D.resid) D.resid[L.i] += solve_residual(T, L, X);
  integrate(T, X);
  float w = loss_weight(T, t + 1, D.hz[L.i]);
  return w != 0.f ? w * loss_value(T, L, X) : 0.f;
}
