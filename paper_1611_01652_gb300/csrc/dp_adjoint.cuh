// Reverse mode of one step of the rigid-body engine (arXiv 1611.01652, section 2.1.1:
// back-propagation through time of the unrolled simulation), written by hand stage by stage.
// Branch rule: clamps, min/max and activation tests take the branch the forward pass took;
// activation masks carry no derivative (the paper's branchless formulation); bfloat16 rounding
// of the controller is straight-through.
#pragma once
#include "dp_forward.cuh"

// Row-adjoint accumulators kept in shared memory per slot (the solver's inner quantities).
enum { RC_LIN = 0, RC_ANGA = 3, RC_ANGB = 6, RC_MEFF = 9, RC_BIAS = 10, RC_BND = 11, RC_N = 12 };

template <class RV>
struct BLaneT {
  LaneT<RV> L;
  SL X0;        // x_t (on chip)
  GL G;         // parameter gradients [field][Bp]
  GC vminus;    // velocities after the external impulses [nb*6][Bp]
};

// R += a b^T for a 3x3 block of the state adjoint at field base (row-major).
__device__ __forceinline__ void add_outer(const SL& XB, int base, float3 a, float3 b) {
  XB[base + 0] += a.x * b.x; XB[base + 1] += a.x * b.y; XB[base + 2] += a.x * b.z;
  XB[base + 3] += a.y * b.x; XB[base + 4] += a.y * b.y; XB[base + 5] += a.y * b.z;
  XB[base + 6] += a.z * b.x; XB[base + 7] += a.z * b.y; XB[base + 8] += a.z * b.z;
}
template <class XV>
__device__ __forceinline__ M3 loadRg(const XV& X, int base) {
  return loadRv(X, base);
}
template <class XV>
__device__ __forceinline__ M3 body_Rg(const XV& X, int b) { return b >= 0 ? loadRv(X, 18 * b) : eye3(); }

// ---------------------------------------------------------------- loss (Eq. L) reverse
// Adds wgt * dl(x)/dx at state X (on-chip) into XB, and the loss point / target gradients.
template <class RV>
__device__ void loss_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& X, const SL& XB, float wgt) {
  if (wgt == 0.f) return;
  const int b = T.loss_body;
  M3 R = loadR(X, 18 * b);
  float3 c = B.L.P.v3(T.o_loss_point), y = B.L.P.v3(T.o_loss_target);
  float3 q = X.v3(18 * b) + mv(R, c);
  float3 gq, gy;
  switch (T.loss_kind) {
    case 0: gq = 2.f * (q - y); gy = -gq; break;
    case 1: { float3 d = q - y; float n = sqrtf(dot3(d, d)); gq = (n > 0.f ? 1.f / n : 0.f) * d; gy = -gq; break; }
    default: gq = y; gy = q; break;
  }
  gq = wgt * gq;
  XB.a3(18 * b, gq);
  add_outer(XB, 18 * b + 3, gq, c);
  B.G.red3(T.o_loss_point, mtv(R, gq));
  B.G.red3(T.o_loss_target, wgt * gy);
}

// ---------------------------------------------------------------- integrate + Eq. 1 reverse
// XB holds the adjoint of x_{t+1}; on return its p/R fields hold the adjoint of x_t's p/R,
// its v/w fields are zero, and VB holds the adjoint of the solver's output velocities.
// (bmask: the bodies to process, bit b)
__device__ inline void integrate_reverse(const DevTopo& T, const GC& Xt, const SL& X, const SL& XB, const SL& VB,
                                  uint32_t bmask = 0xffffffffu) {
  const float h = T.dt;
  for (int b = 0; b < T.nb; ++b) {
    if (!((bmask >> b) & 1u)) continue;
    M3 R = loadRg(Xt, 18 * b);
    float3 w = X.v3(18 * b + 15);  // solver output angular velocity
    M3 A;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.m[j] = R.m[j] + h * (-w.z * R.m[3 + j] + w.y * R.m[6 + j]);
      A.m[3 + j] = R.m[3 + j] + h * (w.z * R.m[j] - w.x * R.m[6 + j]);
      A.m[6 + j] = R.m[6 + j] + h * (-w.y * R.m[j] + w.x * R.m[3 + j]);
    }
    M3 G;
#pragma unroll
    for (int k = 0; k < 9; ++k) G.m[k] = XB[18 * b + 3 + k];
    // R' = (3A - A A^T A)/2  =>  Abar = (3G - (G A^T A + A G^T A + A A^T G))/2
    M3 At = mT(A);
    M3 AtA = mm(At, A);
    M3 t1 = mm(G, AtA), t2 = mm(A, mm(mT(G), A)), t3 = mm(A, mm(At, G));
    M3 Ab;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ab.m[k] = 0.5f * (3.f * G.m[k] - (t1.m[k] + t2.m[k] + t3.m[k]));
    // A = R + h [w]x R
    M3 Wx = {{0.f, -w.z, w.y, w.z, 0.f, -w.x, -w.y, w.x, 0.f}};
    M3 WA = mm(Wx, Ab);
    M3 Om = mm(Ab, mT(R));  // dL/d[w]x = h Abar R^T
    float3 wbar = XB.v3(18 * b + 15) + h * f3(Om.m[7] - Om.m[5], Om.m[2] - Om.m[6], Om.m[3] - Om.m[1]);
    float3 vbar = XB.v3(18 * b + 12) + h * XB.v3(18 * b);
#pragma unroll
    for (int k = 0; k < 9; ++k) XB[18 * b + 3 + k] = Ab.m[k] - h * WA.m[k];
    VB.s3(6 * b, vbar);
    VB.s3(6 * b + 3, wbar);
    XB.s3(18 * b + 12, f3(0.f, 0.f, 0.f));
    XB.s3(18 * b + 15, f3(0.f, 0.f, 0.f));
  }
}

// ---------------------------------------------------------------- PGS reverse
// Replays every sweep backwards. Working velocities are reset to the stored post-sweep values at
// each sweep boundary and un-applied row by row. S[sm_lam] holds the impulse adjoints.
template <class RV>
__device__ void pgs_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& VW, const SL& VB, const SL& RC,
                            const TapeStep& tp) {
  const LaneT<RV>& L = B.L;
  const SL& S = L.S;
  const int Bp = T.Bp;
  for (int s = 0; s < T.nslots; ++s) S[T.sm_lam + s] = 0.f;
  for (int it = T.iters - 1; it >= 0; --it) {
    {
      const float* vi = tp.viter + it * T.nb * 6 * 32;
      for (int b = 0; b < T.nb; ++b)
#pragma unroll
        for (int k = 0; k < 6; ++k) VW[6 * b + k] = vi[(6 * b + k) * 32];
    }
    for (int oi = T.nslots - 1; oi >= 0; --oi) {
      const int s = T.order[oi];
      const RV R = L.rows.at(s * RF_N);
      const float meff = R[RF_MEFF];
      if (!__any_sync(FULLMASK, meff != 0.f)) continue;
      const int kind = T.skind[s], a = T.sa[s], b = T.sb[s];
      const float3 lin = R.v3(RF_LIN);
      const float3 angA = R.v3(RF_ANGA), angB = R.v3(RF_ANGB);
      const float bias = R[RF_BIAS];
      const int o = (it * T.nslots + s) * 32;
      const float la = tp.lam[o];
      const float lb = it > 0 ? tp.lam[o - T.nslots * 32] : (T.ws ? tp.lam0[s * 32] : 0.f);
      const int br = tp.br[o];
      const float dl = la - lb;
      float3 va = f3(0.f, 0.f, 0.f), wa = va, vb = va, wb = va, vba = va, wba = va, vbb = va, wbb = va;
      float ima = 0.f, imb = 0.f;
      float3 IA = f3(0.f, 0.f, 0.f), IB = IA;
      float dbar = 0.f;
      if (a >= 0) {
        ima = S[T.sm_invm + a];
        IA = R.v3(RF_IA);
        va = VW.v3(6 * a) - (dl * ima) * lin;
        wa = VW.v3(6 * a + 3) - dl * IA;
        VW.s3(6 * a, va);
        VW.s3(6 * a + 3, wa);
        vba = VB.v3(6 * a);
        wba = VB.v3(6 * a + 3);
        dbar += ima * dot3(lin, vba) + dot3(IA, wba);
      }
      if (b >= 0) {
        imb = S[T.sm_invm + b];
        IB = R.v3(RF_IB);
        vb = VW.v3(6 * b) + (dl * imb) * lin;
        wb = VW.v3(6 * b + 3) - dl * IB;
        VW.s3(6 * b, vb);
        VW.s3(6 * b + 3, wb);
        vbb = VB.v3(6 * b);
        wbb = VB.v3(6 * b + 3);
        dbar += -imb * dot3(lin, vbb) + dot3(IB, wbb);
      }
      // adjoint of v += M^-1 J^T (la - lb)
      float3 linb = dl * (ima * vba - imb * vbb);
      float3 angAb = f3(0.f, 0.f, 0.f), angBb = angAb;
      if (a >= 0) {
        float3 g = dl * wba;  // adjoint of I_a^-1 angA
        float ia[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) ia[q] = S[T.sm_iinv + 6 * a + q];
        angAb += symv(ia, g);
        const int ib9 = T.sm_iinvb + 9 * a;
        S[ib9 + 0] += g.x * angA.x; S[ib9 + 1] += g.x * angA.y; S[ib9 + 2] += g.x * angA.z;
        S[ib9 + 3] += g.y * angA.x; S[ib9 + 4] += g.y * angA.y; S[ib9 + 5] += g.y * angA.z;
        S[ib9 + 6] += g.z * angA.x; S[ib9 + 7] += g.z * angA.y; S[ib9 + 8] += g.z * angA.z;
        S[T.sm_invmb + a] += dl * dot3(lin, vba);
      }
      if (b >= 0) {
        float3 g = dl * wbb;
        float ib[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) ib[q] = S[T.sm_iinv + 6 * b + q];
        angBb += symv(ib, g);
        const int ib9 = T.sm_iinvb + 9 * b;
        S[ib9 + 0] += g.x * angB.x; S[ib9 + 1] += g.x * angB.y; S[ib9 + 2] += g.x * angB.z;
        S[ib9 + 3] += g.y * angB.x; S[ib9 + 4] += g.y * angB.y; S[ib9 + 5] += g.y * angB.z;
        S[ib9 + 6] += g.z * angB.x; S[ib9 + 7] += g.z * angB.y; S[ib9 + 8] += g.z * angB.z;
        S[T.sm_invmb + b] -= dl * dot3(lin, vbb);
      }
      const float lbar_a = S[T.sm_lam + s] + dbar;  // adjoint of the row's new impulse
      float pbar = 0.f;
      const int rc = s * RC_N;
      if (br == 0) {
        pbar = lbar_a;
      } else if (kind == RK_GT || kind == RK_PT) {
        // bound = +-mu * lambda_n (current value of the contact's normal impulse)
        const int ns_ = T.snormal[s];
        const float lnrm = tp.lam[(it * T.nslots + ns_) * 32];
        const float mu = R[RF_BND];
        const float sg = br == 2 ? 1.f : -1.f;
        RC[rc + RC_BND] += sg * lnrm * lbar_a;
        S[T.sm_lam + ns_] += sg * mu * lbar_a;
      } else if (kind == RK_MOTOR) {
        RC[rc + RC_BND] += (br == 2 ? 1.f : -1.f) * lbar_a;  // d/d(tau_max h)
      }
      // pre = lb - meff (Jv + bias + gamma lb) with the velocities before the row
      float Jv = 0.f;
      if (a >= 0) Jv += dot3(lin, va) + dot3(angA, wa);
      if (b >= 0) Jv += dot3(angB, wb) - dot3(lin, vb);
      RC[rc + RC_MEFF] += -pbar * (Jv + bias + T.gamma * lb);
      const float jvb = -meff * pbar;
      RC[rc + RC_BIAS] += jvb;
      if (a >= 0) {
        VB.s3(6 * a, vba + jvb * lin);
        VB.s3(6 * a + 3, wba + jvb * angA);
        linb += jvb * va;
        angAb += jvb * wa;
      }
      if (b >= 0) {
        VB.s3(6 * b, vbb - jvb * lin);
        VB.s3(6 * b + 3, wbb + jvb * angB);
        linb -= jvb * vb;
        angBb += jvb * wb;
      }
      RC.a3(rc + RC_LIN, linb);
      RC.a3(rc + RC_ANGA, angAb);
      RC.a3(rc + RC_ANGB, angBb);
      S[T.sm_lam + s] = -dbar + pbar * (1.f - meff * T.gamma);
    }
  }
}

// Reverse of the warm-start application v += M^-1 J^T lambda0 over the warm-started rows. The
// initial impulses are constants of the step (a starting guess), so only the rows and the
// inverse masses/inertias that carry them receive adjoints; VB (the adjoint of the velocities
// after the application) is also the adjoint of the pre-solve velocities.
template <class RV>
__device__ void ws_apply_reverse(const DevTopo& T, const LaneT<RV>& L, const SL& VB, const SL& RC, const TapeStep& tp) {
  const SL& S = L.S;
  for (int s = 0; s < T.nslots; ++s) {
    const float dl = tp.lam0[s * 32];
    if (dl == 0.f) continue;
    const RV R = L.rows.at(s * RF_N);
    const int a = T.sa[s], b = T.sb[s], rc = s * RC_N;
    const float3 lin = R.v3(RF_LIN);
    float3 linb = f3(0.f, 0.f, 0.f), angAb = linb, angBb = linb;
    if (a >= 0) {
      const float3 vba = VB.v3(6 * a), g = dl * VB.v3(6 * a + 3), angA = R.v3(RF_ANGA);
      const float ima = S[T.sm_invm + a];
      float ia[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ia[q] = S[T.sm_iinv + 6 * a + q];
      linb += (dl * ima) * vba;
      angAb += symv(ia, g);
      add_outer(S, T.sm_iinvb + 9 * a, g, angA);
      S[T.sm_invmb + a] += dl * dot3(lin, vba);
    }
    if (b >= 0) {
      const float3 vbb = VB.v3(6 * b), g = dl * VB.v3(6 * b + 3), angB = R.v3(RF_ANGB);
      const float imb = S[T.sm_invm + b];
      float ib[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ib[q] = S[T.sm_iinv + 6 * b + q];
      linb -= (dl * imb) * vbb;
      angBb += symv(ib, g);
      add_outer(S, T.sm_iinvb + 9 * b, g, angB);
      S[T.sm_invmb + b] -= dl * dot3(lin, vbb);
    }
    RC.a3(rc + RC_LIN, linb);
    RC.a3(rc + RC_ANGA, angAb);
    RC.a3(rc + RC_ANGB, angBb);
  }
}

// ---------------------------------------------------------------- row assembly reverse
__device__ __forceinline__ void addR_outer(const SL& XB, int b, float3 g, float3 c) {
  if (b >= 0) add_outer(XB, 18 * b + 3, g, c);
}

// Pushes the row adjoints (and the effective-mass adjoint) back to positions, rotations, the
// solver's input velocities (restitution), hinge axes/angles, servo targets and parameters.
template <class RV>
__device__ void rows_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& XB, const SL& VB, const SL& RC) {
  const LaneT<RV>& L = B.L;
  const SL& S = L.S;
  const float h = T.dt;
  const float bh = T.beta / h;
  const float3 ez = f3(0.f, 0.f, 1.f);
  for (int s = 0; s < T.nslots; ++s) {
    const RV R = L.rows.at(s * RF_N);
    const float meff = R[RF_MEFF];
    if (meff == 0.f) continue;  // inactive on this lane: constant row
    const int kind = T.skind[s], idx = T.sidx[s], sub = T.ssub[s], a = T.sa[s], b = T.sb[s];
    const int rc = s * RC_N;
    const float3 lin = R.v3(RF_LIN);
    const float3 angA = R.v3(RF_ANGA), angB = R.v3(RF_ANGB);
    float3 linb = RC.v3(rc + RC_LIN), angAb = RC.v3(rc + RC_ANGA), angBb = RC.v3(rc + RC_ANGB);
    const float biasb = RC[rc + RC_BIAS];
    // effective mass 1/(K + gamma)
    const float Kb = -meff * meff * RC[rc + RC_MEFF];
    if (a >= 0) {
      const float ima = S[T.sm_invm + a];
      linb += (2.f * Kb * ima) * lin;
      angAb += (2.f * Kb) * R.v3(RF_IA);
      const int ib9 = T.sm_iinvb + 9 * a;
      S[ib9 + 0] += Kb * angA.x * angA.x; S[ib9 + 1] += Kb * angA.x * angA.y; S[ib9 + 2] += Kb * angA.x * angA.z;
      S[ib9 + 3] += Kb * angA.y * angA.x; S[ib9 + 4] += Kb * angA.y * angA.y; S[ib9 + 5] += Kb * angA.y * angA.z;
      S[ib9 + 6] += Kb * angA.z * angA.x; S[ib9 + 7] += Kb * angA.z * angA.y; S[ib9 + 8] += Kb * angA.z * angA.z;
      S[T.sm_invmb + a] += Kb * dot3(lin, lin);
    }
    if (b >= 0) {
      const float imb = S[T.sm_invm + b];
      linb += (2.f * Kb * imb) * lin;
      angBb += (2.f * Kb) * R.v3(RF_IB);
      const int ib9 = T.sm_iinvb + 9 * b;
      S[ib9 + 0] += Kb * angB.x * angB.x; S[ib9 + 1] += Kb * angB.x * angB.y; S[ib9 + 2] += Kb * angB.x * angB.z;
      S[ib9 + 3] += Kb * angB.y * angB.x; S[ib9 + 4] += Kb * angB.y * angB.y; S[ib9 + 5] += Kb * angB.y * angB.z;
      S[ib9 + 6] += Kb * angB.z * angB.x; S[ib9 + 7] += Kb * angB.z * angB.y; S[ib9 + 8] += Kb * angB.z * angB.z;
      S[T.sm_invmb + b] += Kb * dot3(lin, lin);
    }
    switch (kind) {
      case RK_JLIN: {
        float3 e = f3(sub == 0 ? 1.f : 0.f, sub == 1 ? 1.f : 0.f, sub == 2 ? 1.f : 0.f);
        float3 anca = L.P.v3(T.o_anchor + 6 * idx), ancb = L.P.v3(T.o_anchor + 6 * idx + 3);
        float3 Cb = (bh * biasb) * e;
        // angA = ra x e, angB = -(rb x e), C = pa + ra - pb - rb
        float3 rab = cross3(e, angAb) + Cb;
        float3 rbb = -cross3(e, angBb) - Cb;
        if (a >= 0) {
          M3 Ra = loadRg(B.X0, 18 * a);
          XB.a3(18 * a, Cb);
          add_outer(XB, 18 * a + 3, rab, anca);
          B.G.red3(T.o_anchor + 6 * idx, mtv(Ra, rab));
        } else {
          B.G.red3(T.o_anchor + 6 * idx, rab);
        }
        M3 Rb = loadRg(B.X0, 18 * b);
        XB.a3(18 * b, -Cb);
        add_outer(XB, 18 * b + 3, rbb, ancb);
        B.G.red3(T.o_anchor + 6 * idx + 3, mtv(Rb, rbb));
        break;
      }
      case RK_JANG: {
        float3 t1, t2;
        onb3(L.P.v3(T.o_axis + 6 * idx), t1, t2);
        float3 tau = sub == 0 ? t1 : t2;
        M3 Ra = body_Rg(B.X0, a), Rb = loadRg(B.X0, 18 * b);
        float3 t = mv(Ra, tau);
        float3 axb = L.P.v3(T.o_axis + 6 * idx + 3);
        float3 ub = mv(Rb, axb);
        float3 ua = S.v3(T.sm_ua + 3 * idx);
        float3 cr = cross3(ub, ua);
        float3 tb = angAb - angBb + (bh * biasb) * cr;
        if (a < 0) tb = -angBb + (bh * biasb) * cr;
        float3 crb = (bh * biasb) * t;
        float3 ubb = cross3(ua, crb);    // c = ub x ua
        float3 uab = cross3(crb, ub);
        S.a3(T.sm_uab + 3 * idx, uab);
        addR_outer(XB, a, tb, tau);
        add_outer(XB, 18 * b + 3, ubb, axb);
        break;
      }
      case RK_LIMIT: {
        float th = S[T.sm_th + idx];
        float lo_j = L.P[T.o_limit + 2 * idx];
        float3 uab;
        if (th <= lo_j) {  // angA = -ua, angB = ua, bias = bh (th - lo)
          uab = angBb - (a >= 0 ? angAb : f3(0.f, 0.f, 0.f));
          S[T.sm_thb + idx] += bh * biasb;
          B.G.red(T.o_limit + 2 * idx, -(bh * biasb));
        } else {           // angA = ua, angB = -ua, bias = bh (hi - th)
          uab = (a >= 0 ? angAb : f3(0.f, 0.f, 0.f)) - angBb;
          S[T.sm_thb + idx] -= bh * biasb;
          B.G.red(T.o_limit + 2 * idx + 1, bh * biasb);
        }
        S.a3(T.sm_uab + 3 * idx, uab);
        break;
      }
      case RK_MOTOR: {
        S.a3(T.sm_uab + 3 * idx, angBb - (a >= 0 ? angAb : f3(0.f, 0.f, 0.f)));
        S[T.sm_wstb + idx] -= biasb;
        B.G.red(T.o_motor + 3 * idx + 1, h * RC[rc + RC_BND]);
        break;
      }
      case RK_GN:
      case RK_GT: {
        M3 Ra = loadRg(B.X0, 18 * a);
        float3 off = L.P.v3(T.o_sph_off + 3 * idx);
        float3 c = mv(Ra, off);
        float rad = L.P[T.o_sph_rad + idx];
        float d = (B.X0[18 * a + 2] + c.z) - rad - T.ground_z;
        float3 ra = c - rad * ez;
        float db = 0.f;
        if (kind == RK_GN) {
          float3 vm = B.vminus.v3(6 * a), wm = B.vminus.v3(6 * a + 3);
          float vn = dot3(lin, vm) + dot3(angA, wm);
          if (d + T.slop < 0.f) db += bh * biasb;
          if (vn < 0.f) {
            float e = L.P[T.o_sph_e + idx];
            B.G.red(T.o_sph_e + idx, vn * biasb);
            float vnb = e * biasb;
            VB.a3(6 * a, vnb * lin);
            VB.a3(6 * a + 3, vnb * angA);
            angAb += vnb * wm;
          }
        } else {
          B.G.red(T.o_sph_mu + idx, RC[rc + RC_BND]);
        }
        float3 rab = cross3(lin, angAb);  // angA = ra x lin (lin constant)
        float3 cb = rab + f3(0.f, 0.f, db);
        float radb = -rab.z - db;
        XB[18 * a + 2] += db;
        add_outer(XB, 18 * a + 3, cb, off);
        B.G.red3(T.o_sph_off + 3 * idx, mtv(Ra, cb));
        B.G.red(T.o_sph_rad + idx, radb);
        break;
      }
      case RK_PN:
      case RK_PT: {
        const int k = T.pk[idx], l = T.pl[idx];
        M3 Ra = loadRg(B.X0, 18 * a), Rb = loadRg(B.X0, 18 * b);
        float3 offk = L.P.v3(T.o_sph_off + 3 * k), offl = L.P.v3(T.o_sph_off + 3 * l);
        float3 ck = mv(Ra, offk), cl = mv(Rb, offl);
        float3 dl = (B.X0.v3(18 * a) + ck) - (B.X0.v3(18 * b) + cl);
        float dist = sqrtf(dot3(dl, dl));
        bool deg = !(dist > 1e-9f);
        float3 n = deg ? ez : (1.f / dist) * dl;
        float rk = L.P[T.o_sph_rad + k], rl = L.P[T.o_sph_rad + l];
        float d = dist - rk - rl;
        float3 ra = ck - rk * n, rb = cl + rl * n;
        float3 nb = f3(0.f, 0.f, 0.f);
        float distb = 0.f, rkb = 0.f, rlb = 0.f;
        if (kind == RK_PN) {
          float3 vma = B.vminus.v3(6 * a), wma = B.vminus.v3(6 * a + 3);
          float3 vmb = B.vminus.v3(6 * b), wmb = B.vminus.v3(6 * b + 3);
          float vn = dot3(n, vma - vmb) + dot3(angA, wma) + dot3(angB, wmb);
          if (d + T.slop < 0.f) distb += bh * biasb;
          if (vn < 0.f) {
            float ek = L.P[T.o_sph_e + k], el = L.P[T.o_sph_e + l];
            float e = ek >= el ? ek : el;
            B.G.red(T.o_sph_e + (ek >= el ? k : l), vn * biasb);
            float vnb = e * biasb;
            nb += vnb * (vma - vmb);
            VB.a3(6 * a, vnb * n);
            VB.a3(6 * b, -vnb * n);
            VB.a3(6 * a + 3, vnb * angA);
            VB.a3(6 * b + 3, vnb * angB);
            angAb += vnb * wma;
            angBb += vnb * wmb;
          }
          nb += linb;
          // angA = ra x n, angB = -(rb x n)
          float3 rab = cross3(n, angAb), rbb = -cross3(n, angBb);
          nb += cross3(angAb, ra) - cross3(angBb, rb);
          // ra = ck - rk n, rb = cl + rl n
          rkb -= dot3(rab, n); nb -= rk * rab;
          rlb += dot3(rbb, n); nb += rl * rbb;
          rkb -= distb; rlb -= distb;  // d = dist - rk - rl
          float3 ckb = rab, clb = rbb;
          float3 dlb = deg ? f3(0.f, 0.f, 0.f) : distb * n + (1.f / dist) * (nb - dot3(n, nb) * n);
          ckb += dlb; clb -= dlb;
          XB.a3(18 * a, dlb); XB.a3(18 * b, -dlb);
          add_outer(XB, 18 * a + 3, ckb, offk);
          add_outer(XB, 18 * b + 3, clb, offl);
          B.G.red3(T.o_sph_off + 3 * k, mtv(Ra, ckb));
          B.G.red3(T.o_sph_off + 3 * l, mtv(Rb, clb));
          B.G.red(T.o_sph_rad + k, rkb);
          B.G.red(T.o_sph_rad + l, rlb);
        } else {
          float3 t1, t2;
          onb3(n, t1, t2);
          float3 t = sub == 0 ? t1 : t2;
          float3 tb = linb + cross3(angAb, ra) - cross3(angBb, rb);
          float3 rab = cross3(t, angAb), rbb = -cross3(t, angBb);
          nb += deg ? f3(0.f, 0.f, 0.f) : onb3_vjp(n, sub == 0 ? tb : f3(0.f, 0.f, 0.f), sub == 1 ? tb : f3(0.f, 0.f, 0.f));
          rkb -= dot3(rab, n); nb -= rk * rab;
          rlb += dot3(rbb, n); nb += rl * rbb;
          float3 ckb = rab, clb = rbb;
          float3 dlb = deg ? f3(0.f, 0.f, 0.f) : (1.f / dist) * (nb - dot3(n, nb) * n);
          ckb += dlb; clb -= dlb;
          XB.a3(18 * a, dlb); XB.a3(18 * b, -dlb);
          add_outer(XB, 18 * a + 3, ckb, offk);
          add_outer(XB, 18 * b + 3, clb, offl);
          B.G.red3(T.o_sph_off + 3 * k, mtv(Ra, ckb));
          B.G.red3(T.o_sph_off + 3 * l, mtv(Rb, clb));
          B.G.red(T.o_sph_rad + k, rkb);
          B.G.red(T.o_sph_rad + l, rlb);
          float muk = L.P[T.o_sph_mu + k], mul = L.P[T.o_sph_mu + l];
          float mu = sqrtf(muk * mul);
          float mub = RC[rc + RC_BND];
          if (mu > 0.f) {
            B.G.red(T.o_sph_mu + k, mub * mul / (2.f * mu));
            B.G.red(T.o_sph_mu + l, mub * muk / (2.f * mu));
          }
        }
        break;
      }
    }
  }
}

// ---------------------------------------------------------------- external impulses reverse
// VB holds the adjoint of the velocities after gravity/gyroscopic impulses; adds into XB
// (x_t's v, w, R) and the mass/inertia gradients. IINVB/INVMB hold the world inverse-inertia
// and inverse-mass adjoints gathered from the solver and the rows.
template <class RV>
__device__ void external_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& XB, const SL& VB,
                                 uint32_t bmask = 0xffffffffu) {
  const SL& S = B.L.S;
  const float h = T.dt;
  for (int b = 0; b < T.nb; ++b)  // the bodies' inertia and mass parameter lines into L1
    if ((bmask >> b) & 1u) {
      for (int k = 0; k < 3; ++k) prefetch_l1(B.L.P.p + (size_t)(T.o_inertia + 3 * b + k) * B.L.P.s);
      prefetch_l1(B.L.P.p + (size_t)(T.o_mass + b) * B.L.P.s);
    }
  for (int b = 0; b < T.nb; ++b) {
    if (!((bmask >> b) & 1u)) continue;
    M3 R = loadRg(B.X0, 18 * b);
    float3 I = B.L.P.v3(T.o_inertia + 3 * b);
    float3 Ii = f3(1.f / I.x, 1.f / I.y, 1.f / I.z);
    float m = B.L.P[T.o_mass + b];
    float iw[6], ii[6];
    rot_diag6(R, I, iw);
    rot_diag6(R, Ii, ii);
    float3 w = B.X0.v3(18 * b + 15);
    float3 z = symv(iw, w);
    float3 gy = -cross3(w, z);
    float3 wmb = VB.v3(6 * b + 3);
    // w- = w + h Iinv gy
    M3 Gi;  // adjoint of Iinv (full 3x3)
#pragma unroll
    for (int k = 0; k < 9; ++k) Gi.m[k] = S[T.sm_iinvb + 9 * b + k];
    Gi.m[0] += h * wmb.x * gy.x; Gi.m[1] += h * wmb.x * gy.y; Gi.m[2] += h * wmb.x * gy.z;
    Gi.m[3] += h * wmb.y * gy.x; Gi.m[4] += h * wmb.y * gy.y; Gi.m[5] += h * wmb.y * gy.z;
    Gi.m[6] += h * wmb.z * gy.x; Gi.m[7] += h * wmb.z * gy.y; Gi.m[8] += h * wmb.z * gy.z;
    float3 gyb = h * symv(ii, wmb);
    float3 wb = wmb - cross3(z, gyb);
    float3 zb = cross3(w, gyb);
    wb += symv(iw, zb);
    // Gw = adjoint of Iw = zb w^T
    M3 Gw = {{zb.x * w.x, zb.x * w.y, zb.x * w.z, zb.y * w.x, zb.y * w.y, zb.y * w.z, zb.z * w.x, zb.z * w.y, zb.z * w.z}};
    // R diag(d) R^T reverse: Rbar += (G + G^T) R diag(d), dbar_k = (R^T G R)_kk
    M3 Rb;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float di = c == 0 ? Ii.x : (c == 1 ? Ii.y : Ii.z);
        float dw = c == 0 ? I.x : (c == 1 ? I.y : I.z);
        float si = 0.f, sw = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          si += (Gi.m[3 * r + q] + Gi.m[3 * q + r]) * R.m[3 * q + c];
          sw += (Gw.m[3 * r + q] + Gw.m[3 * q + r]) * R.m[3 * q + c];
        }
        Rb.m[3 * r + c] = si * di + sw * dw;
      }
    float Ib[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float di = 0.f, dw = 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          di += R.m[3 * r + k] * Gi.m[3 * r + c] * R.m[3 * c + k];
          dw += R.m[3 * r + k] * Gw.m[3 * r + c] * R.m[3 * c + k];
        }
      float Ik = k == 0 ? I.x : (k == 1 ? I.y : I.z);
      Ib[k] = dw - di / (Ik * Ik);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) XB[18 * b + 3 + k] += Rb.m[k];
    XB.a3(18 * b + 12, VB.v3(6 * b));
    XB.a3(18 * b + 15, wb);
    B.G.red3(T.o_inertia + 3 * b, f3(Ib[0], Ib[1], Ib[2]));
    B.G.red(T.o_mass + b, -(S[T.sm_invmb + b] / (m * m)));
  }
}

// ---------------------------------------------------------------- servo reverse
template <class RV, class AV>
__device__ void servo_reverse(const DevTopo& T, const BLaneT<RV>& B, const AV& u, const AV& ubd, const SL& ub) {
  const SL& S = B.L.S;
  const int nout = T.n_layers > 0 ? T.widths[T.n_layers] : 0;
  for (int o = 0; o < nout; ++o) ub[o] = 0.f;
  for (int m = 0; m < T.n_motors; ++m) {
    int j = T.motor_joint[m];
    float g = S[T.sm_wstb + j];
    float br = S[T.sm_wbr + j];
    if (br == 0.f) {
      float k = B.L.P[T.o_motor + 3 * j];
      float um = (m < nout) ? u[m] : 0.f;
      if (m < nout) ub[m] = k * g;
      S[T.sm_thb + j] -= k * g;
      B.G.red(T.o_motor + 3 * j, (um - S[T.sm_th + j]) * g);
    } else {
      B.G.red(T.o_motor + 3 * j + 2, (br == 2.f ? 1.f : -1.f) * g);
    }
  }
  for (int o = 0; o < nout; ++o) ubd[o] = ub[o];
}

// One dense layer reversed on this lane: in_bar[i] (+)= sum_o W[o][i] out_bar[o], using the
// [out][in_pad] weight copy; the ReLU mask of the input is applied when `mask` is set.
template <class AVD, class AVA, class AVI>
__device__ void dense_bwd(const float* __restrict__ Wn, int ni, int no, const AVD& outb, const AVA& in_act,
                          const AVI& inb, bool mask, bool accumulate) {
  const int nip = (ni + 7) & ~7;
  for (int i0 = 0; i0 < ni; i0 += 8) {
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    for (int o = 0; o < no; ++o) {
      float g = outb[o];
      float4 w0 = __ldg(reinterpret_cast<const float4*>(Wn + (size_t)o * nip + i0));
      float4 w1 = __ldg(reinterpret_cast<const float4*>(Wn + (size_t)o * nip + i0 + 4));
      acc[0] = fmaf(w0.x, g, acc[0]); acc[1] = fmaf(w0.y, g, acc[1]);
      acc[2] = fmaf(w0.z, g, acc[2]); acc[3] = fmaf(w0.w, g, acc[3]);
      acc[4] = fmaf(w1.x, g, acc[4]); acc[5] = fmaf(w1.y, g, acc[5]);
      acc[6] = fmaf(w1.z, g, acc[6]); acc[7] = fmaf(w1.w, g, acc[7]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (i0 + k < ni) {
        float v = acc[k];
        if (mask && !(in_act[i0 + k] > 0.f)) v = 0.f;
        inb[i0 + k] = accumulate ? inb[i0 + k] + v : v;
      }
    }
  }
}

// Controller reverse: zb0 holds u_bar (the adjoint of the linear output) on entry. The adjoint
// of each layer's pre-activation output is formed on chip (ping-pong buffers zb0/zb1) and also
// stored in the dump (del[l]) for the weight-gradient reduction. Leaves the input adjoint in sbar.
template <class AV>
__device__ void controller_reverse(const DevTopo& T, const DevPtrs& D, const AV* act, const AV* del, const SL& zb0,
                                   const SL& zb1, const SL& sbar) {
  const int L = T.n_layers;
  SL cur = zb0, nxt = zb1;
  for (int l = L - 1; l >= 0; --l) {
    const int ni = T.widths[l], no = T.widths[l + 1];
    const float* Wn = D.Wn + T.w_off[l];
    if (l > 0) {
      dense_bwd(Wn, ni, no, cur, act[l], nxt, true, false);
      for (int k = 0; k < ni; ++k) del[l - 1][k] = nxt[k];
      const SL tmp = cur;
      cur = nxt;
      nxt = tmp;
    } else {
      dense_bwd(Wn, ni, no, cur, act[0], sbar, false, false);
    }
  }
  if (T.skip) dense_bwd(D.Wn + T.w_off[L], T.widths[0], T.widths[L], del[L - 1], act[0], sbar, false, true);
}

// Controller reverse on the tensor cores (the networks of controller_forward_tc). zb0 holds u_bar;
// the output delta is already in del[2]. Hidden deltas go to del[1], del[0]; the input adjoint to
// sbar. Rows of the 16-row tiles mt0 .. mt1 - 1 only (two warps may take one each).
template <class Q, class AV>
__device__ void controller_reverse_tc(const DevTopo& T, const DevPtrs& D, const AV* act, const AV* del, const SL& zb0,
                                      const SL& sbar, int mt0 = 0, int mt1 = 2) {
  const __nv_bfloat16* Wc = D.Wtc;
  const AV a1 = act[1], a2 = act[2], e0 = del[0], e1 = del[1];
  __syncwarp();
  ctrl_tc_dispatch<Q>(T, [&](auto HC) {
    constexpr int H = decltype(HC)::value;
    constexpr CtrlTCLayout Lw = ctrl_tc_layout(H, H);
    mlp3_backward<CTRL_TC_KP0, H, H, CTRL_TC_NOP>(
        T.widths[0], T.widths[3], [&](int f, int r) { return zb0.lane_at(f, r); }, Wc + Lw.w3t, Wc + Lw.w2t,
        Wc + Lw.w1t, [&](int l, int f, int r) { return (l == 1 ? a1 : a2).lane_at(f, r) > 0.f; },
        [&](int l, int f, int r, float v) { (l == 1 ? e0 : e1).lane_at(f, r) = v; },
        [&](int f, int r, float v) { sbar.lane_at(f, r) = v; }, mt0, mt1);
  });
  __syncwarp();
}

// Features reverse: sbar -> hinge angle/rate adjoints, IMU body state, loss point/target.
template <class RV, class AV>
__device__ void features_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& XB, const AV& sbar) {
  const SL& S = B.L.S;
  int k = 0;
  if (T.features & 1)
    for (int m = 0; m < T.n_motors; ++m) S[T.sm_thb + T.motor_joint[m]] += sbar[k++];
  if (T.features & 2)
    for (int m = 0; m < T.n_motors; ++m) S[T.sm_thdb + T.motor_joint[m]] += sbar[k++];
  if (T.features & 4) k += 2;
  if (T.features & 8) {
    int b = T.imu_body;
    M3 R = loadRg(B.X0, 18 * b);
    float3 w = B.X0.v3(18 * b + 15);
    float3 gb = f3(sbar[k], sbar[k + 1], sbar[k + 2]);
    float3 wlb = f3(sbar[k + 3], sbar[k + 4], sbar[k + 5]);
    k += 6;
    // g = R^T (0,0,-1)  -> Rbar[2][c] -= gb_c ;  wl = R^T w -> Rbar += w wlb^T, wbar += R wlb
    XB[18 * b + 3 + 6] -= gb.x; XB[18 * b + 3 + 7] -= gb.y; XB[18 * b + 3 + 8] -= gb.z;
    add_outer(XB, 18 * b + 3, w, wlb);
    XB.a3(18 * b + 15, mv(R, wlb));
  }
  if (T.features & 16) {
    int b = T.loss_body;
    M3 R = loadRg(B.X0, 18 * b);
    float3 c = B.L.P.v3(T.o_loss_point);
    float3 qb = f3(sbar[k], sbar[k + 1], sbar[k + 2]);
    k += 3;
    XB.a3(18 * b, qb);
    add_outer(XB, 18 * b + 3, qb, c);
    B.G.red3(T.o_loss_point, mtv(R, qb));
    B.G.red3(T.o_loss_target, -qb);
  }
}

// Hinge kinematics reverse (x_t): axis, angle and rate adjoints to R and w.
template <class RV>
__device__ void hinge_reverse(const DevTopo& T, const BLaneT<RV>& B, const SL& XB) {
  const SL& S = B.L.S;
  for (int j = 0; j < T.nj; ++j) {
    int a = T.ja[j], b = T.jb[j];
    float3 uab = S.v3(T.sm_uab + 3 * j);
    M3 Ra = body_Rg(B.X0, a);
    float3 axa = B.L.P.v3(T.o_axis + 6 * j);
    float3 ua = mv(Ra, axa);
    if (T.jtype[j] == 1) {
      M3 Rb = loadRg(B.X0, 18 * b);
      float3 refa = B.L.P.v3(T.o_ref + 6 * j), refb = B.L.P.v3(T.o_ref + 6 * j + 3);
      float3 wa = mv(Ra, refa), wb = mv(Rb, refb);
      float3 c = cross3(wa, wb);
      float y = dot3(c, ua), x = dot3(wa, wb);
      float thb = S[T.sm_thb + j], thdb = S[T.sm_thdb + j];
      float den = x * x + y * y;
      float yb = thb * x / den, xb = -thb * y / den;
      float3 cb = yb * ua;
      uab += yb * c;
      float3 wab = cross3(wb, cb) + xb * wb;
      float3 wbb = cross3(cb, wa) + xb * wa;
      float3 wA = a >= 0 ? B.X0.v3(18 * a + 15) : f3(0.f, 0.f, 0.f);
      float3 wB = B.X0.v3(18 * b + 15);
      uab += thdb * (wB - wA);
      XB.a3(18 * b + 15, thdb * ua);
      if (a >= 0) XB.a3(18 * a + 15, -thdb * ua);
      addR_outer(XB, a, wab, refa);
      add_outer(XB, 18 * b + 3, wbb, refb);
    }
    addR_outer(XB, a, uab, axa);
  }
}
