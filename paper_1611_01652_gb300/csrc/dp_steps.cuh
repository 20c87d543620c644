// The persistent rollout (forward) and reverse-mode kernel templates (one warp = 32 instances for
// the whole horizon; four warps per 32 instances for the compiled topology's reverse pass).
#pragma once
#include <cuda_runtime.h>

#include <cstdlib>
#include <type_traits>

#include "dp_mw.cuh"

extern __shared__ float g_smem[];

// Dynamic shared memory of a persistent kernel: sm_total units of 32 floats.
#define SM_BYTES(T) ((size_t)(T).sm_total * 32 * sizeof(float))

// ------------------------------------------------------------------------------ forward
__device__ __forceinline__ void copy_state_to_smem(const DevTopo& T, const float* src, int i, const SL& X) {
  for (int f = 0; f < 18 * T.nb; ++f) X[f] = src[(size_t)f * T.Bp + i];
}
__device__ __forceinline__ void copy_state_from_smem(const DevTopo& T, float* dst, int i, const SL& X) {
  for (int f = 0; f < 18 * T.nb; ++f) dst[(size_t)f * T.Bp + i] = X[f];
}

// Persistent forward: each warp advances its 32 instances over `nsteps` steps starting at step
// t0. With rollout != 0 it starts from x0, stores checkpoints every ckpt_every steps and the
// per-instance loss of Eq. L.
template <class RV>
__device__ __forceinline__ RV row_view(const DevTopo& T, const DevPtrs& D, float* sm, int i);
template <>
__device__ __forceinline__ SL row_view<SL>(const DevTopo& T, const DevPtrs& D, float* sm, int i) {
  return SL{sm + T.sm_rows * 32};
}
template <>
__device__ __forceinline__ GL row_view<GL>(const DevTopo& T, const DevPtrs& D, float* sm, int i) {
  return GL{D.rows + i, T.Bp};
}

// Persistent forward: each warp advances its 32 instances over `nsteps` steps starting at step
// t0. With rollout != 0 it starts from x0, stores checkpoints every ckpt_every steps and the
// per-instance loss of Eq. L; with REC it also records every step's solver tape and
// controller activations for the reverse pass.
template <class RV, bool REC, class Q>
__global__ void __launch_bounds__(32, 1) k_forward(const __grid_constant__ DevTopo T, const __grid_constant__ DevPtrs D,
                                                    const float* __restrict__ x0, int t0, int nsteps, int rollout) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  float* sm = g_smem + lane;
  LaneT<RV> L{SL{sm}, GC{D.prm + i, T.Bp}, row_view<RV>(T, D, sm, i), i};
  SL X{sm + T.sm_x * 32};
  SL act[DPK_MAXL + 1];
  for (int l = 0; l <= DPK_MAXL; ++l) act[l] = SL{sm + T.sm_act[l] * 32};
  // rollout 1: a whole rollout from x0; rollout 2: the part of a rollout from step t0 on, from
  // the state and loss the previous part left (from x0 when t0 = 0)
  const bool fresh = rollout == 1 || (rollout == 2 && t0 == 0);
  copy_state_to_smem(T, fresh ? x0 : D.state, i, X);
  // impulses of the previous step (the warm start's lambda_prev): none before a rollout
  for (int s = 0; s < T.nslots; ++s) L.S[T.sm_lam + s] = fresh ? 0.f : D.lam_prev[(size_t)s * T.Bp + i];
  // the controller's recurrent state: h^0 = 0 at the start of a rollout
  for (int k = 0; k < T.n_rec; ++k) L.S[T.sm_h + k] = fresh ? 0.f : D.hrec[(size_t)k * T.Bp + i];
  float loss = (rollout == 2 && !fresh) ? D.loss[i] : 0.f;
  if (fresh && T.loss_kind == 3) loss = -dot3(L.P.v3(T.o_loss_target), loss_point(T, L, X));
  const int B = T.B;
  // a rollout steps the warp to the largest horizon among its instances
  const int nrun = rollout ? max(0, min(nsteps, warp_horizon(D, i) - t0)) : nsteps;
  for (int k = 0; k < nrun; ++k) {
    const int t = t0 + k;
    if (rollout) {
      if (t % D.ckpt_every == 0) {
        copy_state_from_smem(T, D.ckpt + (size_t)(t / D.ckpt_every) * 18 * T.nb * T.Bp, i, X);
        if (D.ckpt_lam)
          for (int s = 0; s < T.nslots; ++s)
            D.ckpt_lam[((size_t)(t / D.ckpt_every) * T.nslots + s) * T.Bp + i] = L.S[T.sm_lam + s];
        if (D.ckpt_h)
          for (int k = 0; k < T.n_rec; ++k)
            D.ckpt_h[((size_t)(t / D.ckpt_every) * T.n_rec + k) * T.Bp + i] = L.S[T.sm_h + k];
      }
      if (D.traj && i < B)
        for (int f = 0; f < 18 * T.nb; ++f) D.traj[((size_t)t * B + i) * 18 * T.nb + f] = X[f];
    }
    // the activity log is per rollout step (rollout parts) or per call step (dp_step)
    uint8_t* ao = (D.active && i < B) ? D.active + ((size_t)(rollout == 2 ? t : k) * B + i) * T.nslots : nullptr;
    if (REC)
      loss += step_forward<true, Q>(T, D, L, X, act, t, ao, t,
                                    T.n_layers > 0 && !T.ext_ctrl ? D.dump + (size_t)t * T.Bp + i : nullptr);
    else
      loss += step_forward<false, Q>(T, D, L, X, act, t, ao);
  }
  if (rollout && D.traj && i < B)
    for (int f = 0; f < 18 * T.nb; ++f) D.traj[((size_t)(t0 + nrun) * B + i) * 18 * T.nb + f] = X[f];
  if (T.ext_ctrl && t0 + nrun < T.horizon) {
    // wide controller: input features of the next step, bf16 for the products, and the
    // activation dump column for the weight gradient
    const int tn = t0 + nrun;
    hinge_kinematics(T, L, X);
    controller_features(T, L, X, tn, act[0]);
    __nv_bfloat16* sx = D.s_ext + (size_t)i * T.ext_k0p;
    const size_t N = (size_t)T.horizon * T.Bp;
    for (int k = 0; k < T.ext_k0p; ++k) {
      const float v = k < T.widths[0] ? act[0][k] : 0.f;
      sx[k] = __float2bfloat16_rn(v);
      if (REC && k < T.widths[0]) D.dump[(size_t)(T.dump_act[0] + k) * N + (size_t)tn * T.Bp + i] = v;
    }
  }
  for (int s = 0; s < T.nslots; ++s) D.lam_prev[(size_t)s * T.Bp + i] = L.S[T.sm_lam + s];
  for (int k = 0; k < T.n_rec; ++k) D.hrec[(size_t)k * T.Bp + i] = L.S[T.sm_h + k];
  copy_state_from_smem(T, D.state, i, X);
  bool bad = !isfinite(loss);
  for (int f = 0; f < 18 * T.nb; ++f) bad |= !isfinite(X[f]);
  if (rollout) D.loss[i] = loss;
  if (bad && i < B) D.status[i] |= DPK_ST_NAN_STATE;
}

// The one-warp warm start with the solver tape, out of line (it runs on one warp of k_forward_mw
// and keeps the network's registers out of that kernel's budget).
static __device__ __noinline__ void warm_start_call(const DevTopo& T, const DevPtrs& D, const LaneT<SL>& L, const SL& X,
                                             const TapeStep& tp) {
  warm_start<true>(T, D, L, X, tp);
}

// Persistent rollout of the compiled topology with the solver tape, on four warps per group of
// 32 instances (one CTA per group; a lane is an instance in every warp, as in k_forward). The
// stages outside the sweeps are split: warp w takes the joints and bodies it owns
// (DevTopo.mw_jmask, mw_bmask: kinematics, servo targets, external impulses, the warm start's
// application, integration), every fourth constraint slot of the row assembly and every fourth
// field of the tape and checkpoint copies; warps 0 and 1 take one 16-row tile each of the
// tensor-core controller's products. The sweeps, the controller's features and the loss run on
// warp 0. Each quantity is computed by the same arithmetic in the same order as in k_forward,
// so the two kernels give identical results. For rollouts (rollout != 0) without the harvest or
// gait noise; with the wide controller (one step per launch) the step's controller output comes
// from the batched products and the next step's input features go back to them, as in
// k_forward.
template <class Q>
__global__ void __launch_bounds__(128, 1) k_forward_mw(const __grid_constant__ DevTopo T, const __grid_constant__ DevPtrs D,
                                                       const float* __restrict__ x0, int t0, int nsteps, int rollout) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int Bp = T.Bp, B = T.B, nf = 18 * T.nb;
  float* sm = g_smem + lane;
  LaneT<SL> L{SL{sm}, GC{D.prm + i, Bp}, SL{sm + T.sm_rows * 32}, i};
  const SL X{sm + T.sm_x * 32};
  SL act[DPK_MAXL + 1];
  for (int l = 0; l <= DPK_MAXL; ++l) act[l] = SL{sm + T.sm_act[l] * 32};
  const uint32_t bm = T.mw_bmask[warp], jm = T.mw_jmask[warp];
  const bool fresh = rollout == 1 || (rollout == 2 && t0 == 0);
  const float* xs = fresh ? x0 : D.state;
  for (int f = warp; f < nf; f += 4) X[f] = xs[(size_t)f * Bp + i];
  for (int s = warp; s < T.nslots; s += 4) L.S[T.sm_lam + s] = fresh ? 0.f : D.lam_prev[(size_t)s * Bp + i];
  if (warp == 0)
    for (int k = 0; k < T.n_rec; ++k) L.S[T.sm_h + k] = fresh ? 0.f : D.hrec[(size_t)k * Bp + i];
  mw_barrier();
  float loss = (rollout == 2 && !fresh) ? D.loss[i] : 0.f;  // warp 0's copy is the one kept
  if (fresh && T.loss_kind == 3) loss = -dot3(L.P.v3(T.o_loss_target), loss_point(T, L, X));
  const int nrun = max(0, min(nsteps, warp_horizon(D, i) - t0));
  const size_t N = (size_t)T.horizon * Bp;
  for (int k = 0; k < nrun; ++k) {
    const int t = t0 + k;
    if (t % D.ckpt_every == 0) {
      const size_t c = (size_t)(t / D.ckpt_every);
      for (int f = warp; f < nf; f += 4) D.ckpt[(c * nf + f) * Bp + i] = X[f];
      if (D.ckpt_lam)
        for (int s = warp; s < T.nslots; s += 4) D.ckpt_lam[(c * T.nslots + s) * Bp + i] = L.S[T.sm_lam + s];
      if (D.ckpt_h && warp == 0)
        for (int q = 0; q < T.n_rec; ++q) D.ckpt_h[(c * T.n_rec + q) * Bp + i] = L.S[T.sm_h + q];
    }
    if (D.traj && i < B)
      for (int f = warp; f < nf; f += 4) D.traj[((size_t)t * B + i) * nf + f] = X[f];
    uint8_t* ao = (D.active && i < B) ? D.active + ((size_t)t * B + i) * T.nslots : nullptr;
    // joint kinematics, controller, servo targets
    hinge_kinematics(T, L, X, jm);
    mw_barrier();
    if (T.ext_ctrl) {
      // wide controller: its output for this step was computed between launches
      if (warp == 0) {
        const float* ue = D.u_ext + ((size_t)t * Bp + i) * T.ext_nop;
        for (int m = 0; m < T.widths[T.n_layers]; ++m) act[T.n_layers][m] = ue[m];
      }
      mw_barrier();
      servo_targets(T, L, act[T.n_layers], jm);
    } else if (T.n_layers > 0) {
      float* dump_col = D.dump + (size_t)t * Bp + i;
      if (warp == 0) {
        controller_features(T, L, X, t, act[0]);
        if (T.n_rec) {  // recurrent state h^t: the last inputs
          const int base = T.widths[0] - T.n_rec;
          for (int q = 0; q < T.n_rec; ++q) act[0][base + q] = qz(T, L.S[T.sm_h + q]);
        }
      }
      mw_barrier();
      if (T.mlp_tc) {
        if (warp < 2) ctrl_tc_forward_q<Q, SL>(T, D, act, dump_col, warp, warp + 1);
      } else if (warp == 0) {
        controller_forward(T, D, act);
      }
      mw_barrier();
      if (warp == 0) {
        if (T.n_rec) {  // h^{t+1} = tanh of the last outputs
          const int base = T.widths[T.n_layers] - T.n_rec;
          for (int q = 0; q < T.n_rec; ++q) L.S[T.sm_h + q] = tanhf(act[T.n_layers][base + q]);
        }
        for (int l = 0; l <= T.n_layers; ++l) {
          if (T.mlp_tc && l > 0 && l < T.n_layers) continue;  // hidden layers went straight to the dump
          for (int q = 0; q < T.widths[l]; ++q) dump_col[(size_t)(T.dump_act[l] + q) * N] = act[l][q];
        }
      }
      servo_targets(T, L, act[T.n_layers], jm);
    } else {
      servo_targets(T, L, act[0], jm);
    }
    // external impulses and world inverse inertias; the tape's pre-solve velocities
    external_impulses(T, L, X, bm);
    const TapeStep tp = tape_step(T, D, t);
    for (int b = 0; b < T.nb; ++b)
      if ((bm >> b) & 1u)
#pragma unroll
        for (int q = 0; q < 6; ++q) tp.vminus[(6 * b + q) * 32] = X[18 * b + 12 + q];
    mw_barrier();
    assemble_rows(T, L, X, ao, warp, 4);
    mw_barrier();
    for (int f = warp; f < T.nslots * RF_N; f += 4) tp.rows[f * 32] = L.rows[f];
    if (T.ws) {
      if (T.ws_net) {
        // a learned network's start: the one-warp stage (features, the network on the tensor
        // cores, projection, application to every body) on warp 0, as in k_forward
        if (warp == 0) warm_start_call(T, D, L, X, tp);
      } else {
        warm_start_mw<true>(T, L, X, tp, warp, bm);
      }
    }
    mw_barrier();
    if (warp == 0) {
      pgs_solve_static<Q, true>(T, L, X, tp);
      if (D.resid) D.resid[i] += solve_residual(T, L, X);
    }
    mw_barrier();
    integrate(T, X, bm);
    mw_barrier();
    if (warp == 0) {
      const float w = loss_weight(T, t + 1, D.hz[i]);
      if (w != 0.f) loss += w * loss_value(T, L, X);
    }
  }
  if (D.traj && i < B)
    for (int f = warp; f < nf; f += 4) D.traj[((size_t)(t0 + nrun) * B + i) * nf + f] = X[f];
  if (T.ext_ctrl && t0 + nrun < T.horizon && warp == 0) {
    // wide controller: input features of the next step, bf16 for the products, and the
    // activation dump column for the weight gradient
    const int tn = t0 + nrun;
    hinge_kinematics(T, L, X);
    controller_features(T, L, X, tn, act[0]);
    __nv_bfloat16* sx = D.s_ext + (size_t)i * T.ext_k0p;
    for (int q = 0; q < T.ext_k0p; ++q) {
      const float v = q < T.widths[0] ? act[0][q] : 0.f;
      sx[q] = __float2bfloat16_rn(v);
      if (q < T.widths[0]) D.dump[(size_t)(T.dump_act[0] + q) * N + (size_t)tn * Bp + i] = v;
    }
  }
  for (int s = warp; s < T.nslots; s += 4) D.lam_prev[(size_t)s * Bp + i] = L.S[T.sm_lam + s];
  if (warp == 0)
    for (int q = 0; q < T.n_rec; ++q) D.hrec[(size_t)q * Bp + i] = L.S[T.sm_h + q];
  bool bad = false;
  for (int f = warp; f < nf; f += 4) {
    D.state[(size_t)f * Bp + i] = X[f];
    bad |= !isfinite(X[f]);
  }
  if (warp == 0) {
    bad |= !isfinite(loss);
    D.loss[i] = loss;
  }
  if (bad && i < B) atomicOr(D.status + i, DPK_ST_NAN_STATE);
}

// ------------------------------------------------------------------------------ backward
struct BwdCtx {
  SL S, X, XB, VB, RC, sbar;
  GC P;
  GL G;
  int i;
  float dl;
};

// Per-step views of the reverse pass: the step's tape record, its controller dump columns and the
// lane views built on them.
template <class RV>
struct RevStep {
  TapeStep tp;
  LaneT<RV> L;
  BLaneT<RV> Bl;
  GW act[DPK_MAXL + 1], del[DPK_MAXL + 1];
  SL zb0, zb1;
};
template <class RV>
__device__ __forceinline__ RevStep<RV> rev_views(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, int t, int ts) {
  const int Bp = T.Bp, i = C.i;
  const size_t N = (size_t)T.horizon * Bp;
  const size_t n = (size_t)t * Bp + i;
  const TapeStep tp = tape_step(T, D, ts);
  LaneT<RV> L{C.S, C.P, RV{tp.rows}, i};
  RevStep<RV> V{tp, L, BLaneT<RV>{L, C.X, C.G, GC{tp.vminus, 32}}, {}, {}, SL{C.S.p + T.sm_zb * 32}, SL{nullptr}};
  for (int l = 0; l <= DPK_MAXL; ++l) {
    V.act[l] = GW{D.dump + (size_t)T.dump_act[l] * N + n, N};
    V.del[l] = GW{D.dump + (size_t)T.dump_del[l] * N + n, N};
  }
  if (T.ext_ctrl) V.act[T.n_layers] = GW{D.u_ext + n * T.ext_nop, 1};  // wide controller's output u_t
  int maxw = 1;
  for (int l = 0; l <= T.n_layers && T.n_layers > 0; ++l) maxw = max(maxw, T.widths[l]);
  V.zb1 = SL{C.S.p + (T.sm_zb + maxw) * 32};
  return V;
}

// First part of the reverse of step t (through the zeroing of the solver's adjoint
// accumulators): loss term and integrator with x_{t+1} on chip, then x_t and its per-step
// forward quantities recomputed bit-identically (hinge kinematics, servo targets, inverse
// inertias).
template <class Q, class RV>
__device__ void reverse_step_head(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, const RevStep<RV>& V, int t,
                                  int ts, const float* x_t, const float* x_t1) {
  const int Bp = T.Bp, i = C.i;
  if (ts > 0) prefetch_record_l2(T, tape_step(T, D, ts - 1).rec);  // the next step to reverse
  copy_state_to_smem(T, x_t1, i, C.X);
  if (T.grad_decay != 1.f) {  // section 3.2: the adjoint from later steps shrinks by alpha per step
    for (int f = 0; f < 18 * T.nb; ++f) C.XB[f] *= T.grad_decay;
    for (int k = 0; k < T.n_rec; ++k) C.S[T.sm_hb + k] *= T.grad_decay;  // and so does h's
  }
  loss_reverse(T, V.Bl, C.X, C.XB, loss_weight(T, t + 1, D.hz[i]) * C.dl);
  integrate_reverse(T, GC{x_t + i, Bp}, C.X, C.XB, C.VB);
  copy_state_to_smem(T, x_t, i, C.X);
  hinge_kinematics(T, V.L, C.X);
  servo_targets(T, V.L, V.act[T.n_layers > 0 ? T.n_layers : 0]);
  inverse_inertia(T, V.L, C.X);
  for (int j = 0; j < T.nj; ++j) {
    C.S[T.sm_thb + j] = 0.f; C.S[T.sm_thdb + j] = 0.f; C.S[T.sm_wstb + j] = 0.f;
    C.S.s3(T.sm_uab + 3 * j, f3(0.f, 0.f, 0.f));
  }
  for (int b = 0; b < T.nb; ++b) {
    C.S[T.sm_invmb + b] = 0.f;
    for (int q = 0; q < 9; ++q) C.S[T.sm_iinvb + 9 * b + q] = 0.f;
  }
  for (int q = 0; q < T.nslots * RC_N; ++q) C.RC[q] = 0.f;
}

// The in-step controller's reverse around its products: servo targets and the recurrent
// outputs' tanh (head: u_bar into zb0 and the output delta), then, after the products, the
// features and the recurrent input (tail).
template <class RV>
__device__ void ctrl_reverse_head(const DevTopo& T, const BwdCtx& C, const RevStep<RV>& V) {
  const GW* act = V.act;
  const GW* del = V.del;
  servo_reverse(T, V.Bl, act[T.n_layers], del[T.n_layers - 1], V.zb0);
  if (T.n_rec) {  // adjoint of the recurrent outputs: h^{t+1} = tanh(z)
    const int base = T.widths[T.n_layers] - T.n_rec;
    for (int k = 0; k < T.n_rec; ++k) {
      const float th = tanhf(act[T.n_layers][base + k]);
      const float zb = C.S[T.sm_hb + k] * (1.f - th * th);
      V.zb0[base + k] = zb;
      del[T.n_layers - 1][base + k] = zb;
    }
  }
}
template <class RV>
__device__ void ctrl_reverse_tail(const DevTopo& T, const BwdCtx& C, const RevStep<RV>& V) {
  features_reverse(T, V.Bl, C.XB, C.sbar);
  if (T.n_rec) {  // adjoint of h^t (straight through its bfloat16 rounding), carried to step t - 1
    const int base = T.widths[0] - T.n_rec;
    for (int k = 0; k < T.n_rec; ++k) C.S[T.sm_hb + k] = C.sbar[base + k];
  }
}

// Servo-target, controller, feature and hinge-kinematics reverse of step t (after the
// external impulses' reverse), down to the adjoint of x_t.
template <class Q, class RV>
__device__ void reverse_step_ctrl(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, const RevStep<RV>& V) {
  const int i = C.i;
  const GW* act = V.act;
  const GW* del = V.del;
  if (T.ext_ctrl) {
    // wide controller: the output adjoint goes to the batched products; the features' adjoint
    // comes back into the next launch
    servo_reverse(T, V.Bl, act[T.n_layers], del[T.n_layers - 1], V.zb0);
    float* ub = D.ub_ext + (size_t)i * 16;
    for (int o = 0; o < 16; ++o) ub[o] = o < T.widths[T.n_layers] ? V.zb0[o] : 0.f;
  } else if (T.n_layers > 0) {
    ctrl_reverse_head(T, C, V);
    if (T.mlp_tc)
      controller_reverse_tc<Q>(T, D, act, del, V.zb0, C.sbar);
    else
      controller_reverse(T, D, act, del, V.zb0, V.zb1, C.sbar);
    ctrl_reverse_tail(T, C, V);
  } else {
    servo_reverse(T, V.Bl, act[0], act[0], V.zb0);
  }
  hinge_reverse(T, V.Bl, C.XB);
}

// reverse_step_ctrl on the four warps of k_backward_mw (called by every warp; ends after a CTA
// barrier): warp 0 takes the servo, feature and hinge-kinematics reverse, warps 0 and 1 one
// 16-row tile each of the tensor-core controller's reverse products.
template <class Q, class RV>
__device__ void reverse_step_ctrl_mw(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, const RevStep<RV>& V,
                                     int warp) {
  if (T.ext_ctrl || T.n_layers == 0 || !T.mlp_tc) {
    if (warp == 0) reverse_step_ctrl<Q>(T, D, C, V);
    mw_barrier();
    return;
  }
  if (warp == 0) ctrl_reverse_head(T, C, V);
  mw_barrier();
  if (warp < 2) controller_reverse_tc<Q>(T, D, V.act, V.del, V.zb0, C.sbar, warp, warp + 1);
  mw_barrier();
  if (warp == 0) {
    ctrl_reverse_tail(T, C, V);
    hinge_reverse(T, V.Bl, C.XB);
  }
  mw_barrier();
}

// Last part of the reverse of step t (after the solver's reverse sweeps): warm-start
// application, row assembly, external impulses, then the stages above, down to the adjoint of x_t.
template <class Q, class RV>
__device__ void reverse_step_tail(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, const RevStep<RV>& V) {
  if (T.ws) ws_apply_reverse(T, V.L, C.VB, C.RC, V.tp);
  rows_reverse(T, V.Bl, C.XB, C.VB, C.RC);
  external_reverse(T, V.Bl, C.XB, C.VB);
  reverse_step_ctrl<Q>(T, D, C, V);
}

// Reverse of step t from its tape slot ts, with x_t and x_{t+1} in global memory. RV is the
// tape-row view: read-only (GSR) when the rollout recorded the whole tape, else GS.
template <class Q, class RV>
__device__ void reverse_step(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, int t, int ts, const float* x_t,
                             const float* x_t1) {
  const RevStep<RV> V = rev_views<RV>(T, D, C, t, ts);
  reverse_step_head<Q, RV>(T, D, C, V, t, ts, x_t, x_t1);
  if constexpr (Q::id != 0 && std::is_same<RV, GSR>::value) {
    pgs_reverse_static<Q>(T, V.L, V.tp);
  } else {
    const SL VW{C.S.p + T.sm_vw * 32};
    pgs_reverse(T, V.Bl, VW, C.VB, C.RC, V.tp);
  }
  reverse_step_tail<Q, RV>(T, D, C, V);
}

// Reverse mode through the last rollout, last step first. With a full tape every step is read
// from it; otherwise each checkpoint segment (last first) is recomputed with its tape.
template <class Q>
__global__ void __launch_bounds__(32, 1) k_backward(const __grid_constant__ DevTopo T, const __grid_constant__ DevPtrs D) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  const int Bp = T.Bp;
  const size_t N = (size_t)T.horizon * Bp;
  const int nf = 18 * T.nb;
  float* sm = g_smem + lane;
  BwdCtx C{SL{sm}, SL{sm + T.sm_x * 32}, SL{sm + T.sm_xb * 32}, SL{sm + T.sm_vb * 32}, SL{sm + T.sm_rc * 32},
           SL{sm + T.sm_sbar * 32}, GC{D.prm + i, Bp}, GL{D.grad_prm + i, Bp}, i, D.dloss[i]};
  for (int f = 0; f < nf; ++f) C.XB[f] = 0.f;
  for (int k = 0; k < T.n_rec; ++k) C.S[T.sm_hb + k] = 0.f;  // no adjoint reaches h^T
  const size_t sbytes = (size_t)nf * Bp;
  const int Tw = warp_horizon(D, i);  // the rollout stepped this warp to Tw
  if (D.tape_full) {
    for (int t = Tw - 1; t >= 0; --t)
      reverse_step<Q, GSR>(T, D, C, t, t, D.ckpt + (size_t)t * sbytes, t + 1 < Tw ? D.ckpt + (size_t)(t + 1) * sbytes : D.state);
  } else {
    const int K = D.ckpt_every;
    for (int c = (Tw - 1) / K; c >= 0; --c) {
      const int ta = c * K;
      const int tb = min(Tw, ta + K);
      copy_state_to_smem(T, D.ckpt + (size_t)c * sbytes, i, C.X);
      if (T.ws)  // the previous impulses the segment's first step started from
        for (int s = 0; s < T.nslots; ++s) C.S[T.sm_lam + s] = D.ckpt_lam[((size_t)c * T.nslots + s) * Bp + i];
      for (int k = 0; k < T.n_rec; ++k)  // the controller's recurrent state at the segment's start
        C.S[T.sm_h + k] = D.ckpt_h[((size_t)c * T.n_rec + k) * Bp + i];
      for (int t = ta; t < tb; ++t) {
        copy_state_from_smem(T, D.seg + (size_t)(t - ta) * sbytes, i, C.X);
        const TapeStep tp = tape_step(T, D, t - ta);
        LaneT<GS> L{C.S, C.P, GS{tp.rows}, i};
        const size_t n = (size_t)t * Bp + i;
        GW aw[DPK_MAXL + 1];
        for (int l = 0; l <= DPK_MAXL; ++l) aw[l] = GW{D.dump + (size_t)T.dump_act[l] * N + n, N};
        step_forward<true, Q>(T, D, L, C.X, aw, t, nullptr, t - ta);
      }
      copy_state_from_smem(T, D.seg + (size_t)(tb - ta) * sbytes, i, C.X);
      for (int t = tb - 1; t >= ta; --t)
        reverse_step<Q, GS>(T, D, C, t, t - ta, D.seg + (size_t)(t - ta) * sbytes, D.seg + (size_t)(t - ta + 1) * sbytes);
    }
  }
  if (T.loss_kind == 3) {  // initial term -a.q(x_0) of the displacement loss
    copy_state_to_smem(T, D.ckpt, i, C.X);
    const int b = T.loss_body;
    M3 R = loadR(C.X, 18 * b);
    float3 c = C.P.v3(T.o_loss_point), a = C.P.v3(T.o_loss_target);
    float3 gq = -C.dl * a;
    C.XB.a3(18 * b, gq);
    add_outer(C.XB, 18 * b + 3, gq, c);
    C.G.red3(T.o_loss_point, mtv(R, gq));
    C.G.red3(T.o_loss_target, -C.dl * (C.X.v3(18 * b) + mv(R, c)));
  }
  for (int f = 0; f < nf; ++f) D.grad_state0[(size_t)f * Bp + i] = C.XB[f];
}

// Reverse mode through the last rollout on four warps per group of 32 instances (compiled
// topology, whole tape recorded by the rollout). Every warp runs every phase of a step on its
// share: bodies and joints split by DevTopo.mw_own (state copies, integrator, hinge kinematics,
// servo targets, inverse inertias, warm-start and row-assembly reverse, external impulses),
// the solver's reverse sweeps split into the chain and three helpers (dp_mw.cuh); warp 0 alone
// runs the servo, controller, feature and hinge reverse. The warps meet at CTA barrier 1
// between phases; every warp executes the same barrier sequence. Same arithmetic as
// k_backward up to the order of the row-adjoint sums, which is fixed.
// One step of the four-warp reverse pass (called by every warp of the CTA; ends after a CTA
// barrier): step t from its tape record and x_t from the checkpoints, with x_{t+1} on chip in
// C.X (copied there first from x_t1 when load_x1 is set); the state adjoint in C.XB is that of
// x_{t+1} on entry and that of x_t on exit.
// Step t's state checkpoint and controller activations of this CTA's 32 instances into L2, one
// 128-byte line per field, spread over the CTA's threads (the reverse of step t + 1 runs
// meanwhile).
__device__ __forceinline__ void mw_prefetch_step_l2(const DevTopo& T, const DevPtrs& D, int t) {
  const int Bp = T.Bp, nf = 18 * T.nb, base = blockIdx.x * 32;
  const float* x = D.ckpt + (size_t)t * nf * Bp + base;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) prefetch_l2(x + (size_t)f * Bp);
  // the controller's activation rows (its delta rows are written, not read, by the reverse)
  if (T.n_layers == 0 || T.ext_ctrl) return;
  const size_t N = (size_t)T.horizon * Bp;
  const float* d = D.dump + (size_t)t * Bp + base;
  for (int l = 0; l <= T.n_layers; ++l)
    for (int r = threadIdx.x; r < T.widths[l]; r += blockDim.x) prefetch_l2(d + (size_t)(T.dump_act[l] + r) * N);
}

template <class Q>
__device__ void mw_reverse_step(const DevTopo& T, const DevPtrs& D, const BwdCtx& C, int t, const float* x_t1,
                                bool load_x1, int warp, uint32_t bm, uint32_t jm) {
  const int i = C.i, Bp = T.Bp, nf = 18 * T.nb;
  const size_t sbytes = (size_t)nf * Bp;
  const RevStep<GSR> V = rev_views<GSR>(T, D, C, t, t);
  const float* x_t = D.ckpt + (size_t)t * sbytes;
  if (load_x1)
    for (int f = warp; f < nf; f += 4) C.X[f] = x_t1[(size_t)f * Bp + i];
  if (t > 0) {  // the next step to reverse: its tape record, state checkpoint and controller columns
    if (warp == 0) prefetch_record_l2(T, tape_step(T, D, t - 1).rec);
    mw_prefetch_step_l2(T, D, t - 1);
  }
  if (T.grad_decay != 1.f) {  // section 3.2: the adjoint from later steps shrinks by alpha per step
    for (int f = warp; f < nf; f += 4) C.XB[f] *= T.grad_decay;
    if (warp == 0)
      for (int k = 0; k < T.n_rec; ++k) C.S[T.sm_hb + k] *= T.grad_decay;  // and so does h's
  }
  mw_barrier();
  // loss term (by the loss body's owner) and integrator, x_{t+1} on chip
  if (T.mw_own[T.loss_body] == warp) loss_reverse(T, V.Bl, C.X, C.XB, loss_weight(T, t + 1, D.hz[i]) * C.dl);
  integrate_reverse(T, GC{x_t + i, Bp}, C.X, C.XB, C.VB, bm);
  mw_barrier();
  // x_t on chip; accumulators zeroed
  for (int f = warp; f < nf; f += 4) C.X[f] = x_t[(size_t)f * Bp + i];
  for (int j = 0; j < T.nj; ++j) {
    if (!((jm >> j) & 1u)) continue;
    C.S[T.sm_thb + j] = 0.f; C.S[T.sm_thdb + j] = 0.f; C.S[T.sm_wstb + j] = 0.f;
    C.S.s3(T.sm_uab + 3 * j, f3(0.f, 0.f, 0.f));
  }
  for (int b = 0; b < T.nb; ++b) {
    if (!((bm >> b) & 1u)) continue;
    C.S[T.sm_invmb + b] = 0.f;
    for (int q = 0; q < 9; ++q) C.S[T.sm_iinvb + 9 * b + q] = 0.f;
  }
  for (int q = warp; q < T.nslots * RC_N; q += 4) C.RC[q] = 0.f;
  mw_barrier();
  // per-step forward quantities of x_t, recomputed bit-identically
  hinge_kinematics(T, V.L, C.X, jm);
  servo_targets(T, V.L, V.act[T.n_layers > 0 ? T.n_layers : 0], jm);
  inverse_inertia(T, V.L, C.X, bm);
  mw_barrier();
  pgs_reverse_mw<Q>(T, V.L, V.tp, warp);
  if (T.ws) {
    ws_apply_reverse_own(T, V.L, C.VB, C.RC, V.tp, warp);
    mw_barrier();
  }
  rows_reverse_own(T, V.Bl, C.XB, C.VB, C.RC, warp);
  mw_barrier();
  external_reverse(T, V.Bl, C.XB, C.VB, bm);
  mw_barrier();
  reverse_step_ctrl_mw<Q>(T, D, C, V, warp);
}

// Initial term -a.q(x_0) of the displacement loss (warp 0).
__device__ __forceinline__ void loss_initial_reverse(const DevTopo& T, const DevPtrs& D, const BwdCtx& C) {
  copy_state_to_smem(T, D.ckpt, C.i, C.X);
  const int b = T.loss_body;
  M3 R = loadR(C.X, 18 * b);
  float3 c = C.P.v3(T.o_loss_point), a = C.P.v3(T.o_loss_target);
  float3 gq = -C.dl * a;
  C.XB.a3(18 * b, gq);
  add_outer(C.XB, 18 * b + 3, gq, c);
  C.G.red3(T.o_loss_point, mtv(R, gq));
  C.G.red3(T.o_loss_target, -C.dl * (C.X.v3(18 * b) + mv(R, c)));
}

// Reverse mode through the last rollout on four warps per group of 32 instances (compiled
// topology, whole tape): every step by mw_reverse_step, last first.
template <class Q>
__global__ void __launch_bounds__(128, 1) k_backward_mw(const __grid_constant__ DevTopo T, const __grid_constant__ DevPtrs D) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int Bp = T.Bp;
  const int nf = 18 * T.nb;
  float* sm = g_smem + lane;
  BwdCtx C{SL{sm}, SL{sm + T.sm_x * 32}, SL{sm + T.sm_xb * 32}, SL{sm + T.sm_vb * 32}, SL{sm + T.sm_rc * 32},
           SL{sm + T.sm_sbar * 32}, GC{D.prm + i, Bp}, GL{D.grad_prm + i, Bp}, i, D.dloss[i]};
  const uint32_t bm = T.mw_bmask[warp], jm = T.mw_jmask[warp];
  for (int f = warp; f < nf; f += 4) C.XB[f] = 0.f;
  if (warp == 0)
    for (int k = 0; k < T.n_rec; ++k) C.S[T.sm_hb + k] = 0.f;
  const size_t sbytes = (size_t)nf * Bp;
  const int Tw = warp_horizon(D, i);  // the same for the CTA's four warps (same instances)
  for (int t = Tw - 1; t >= 0; --t) {
    // x_{t+1} is on chip from the previous (later) step, except for the first one reversed
    const float* x_t1 = t + 1 < Tw ? D.ckpt + (size_t)(t + 1) * sbytes : D.state;
    mw_reverse_step<Q>(T, D, C, t, x_t1, t == Tw - 1, warp, bm, jm);
  }
  if (warp != 0) return;
  if (T.loss_kind == 3) loss_initial_reverse(T, D, C);
  for (int f = 0; f < nf; ++f) D.grad_state0[(size_t)f * Bp + i] = C.XB[f];
}

// The wide controller's per-step reverse launches (k_backward_ext) on four warps per group of 32
// instances (compiled topology, whole tape): the feature adjoint of x_{t+1} (joint kinematics split
// by joint owner, the features' and hinges' reverse on warp 0), then mw_reverse_step of step t.
template <class Q>
__global__ void __launch_bounds__(128, 1) k_backward_ext_mw(const __grid_constant__ DevTopo T,
                                                           const __grid_constant__ DevPtrs D, int t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int Bp = T.Bp;
  const int nf = 18 * T.nb;
  float* sm = g_smem + lane;
  BwdCtx C{SL{sm}, SL{sm + T.sm_x * 32}, SL{sm + T.sm_xb * 32}, SL{sm + T.sm_vb * 32}, SL{sm + T.sm_rc * 32},
           SL{sm + T.sm_sbar * 32}, GC{D.prm + i, Bp}, GL{D.grad_prm + i, Bp}, i, D.dloss[i]};
  const uint32_t bm = T.mw_bmask[warp], jm = T.mw_jmask[warp];
  const int Tw = warp_horizon(D, i);  // the same for the CTA's four warps
  if (t >= Tw) return;                // this group's rollout ended before step t
  const size_t sbytes = (size_t)nf * Bp;
  for (int f = warp; f < nf; f += 4) C.XB[f] = D.grad_state0[(size_t)f * Bp + i];
  const int tn = t + 1;
  if (tn < Tw) {  // adjoint of the features of x_{t+1}
    const float* xs = D.ckpt + (size_t)tn * sbytes;
    for (int f = warp; f < nf; f += 4) C.X[f] = xs[(size_t)f * Bp + i];
    mw_barrier();
    LaneT<GSR> L{C.S, C.P, GSR{D.ckpt}, i};
    BLaneT<GSR> Bl{L, C.X, C.G, GC{D.ckpt, 32}};
    hinge_kinematics(T, L, C.X, jm);
    for (int j = 0; j < T.nj; ++j) {
      if (!((jm >> j) & 1u)) continue;
      C.S[T.sm_thb + j] = 0.f; C.S[T.sm_thdb + j] = 0.f; C.S[T.sm_wstb + j] = 0.f;
      C.S.s3(T.sm_uab + 3 * j, f3(0.f, 0.f, 0.f));
    }
    mw_barrier();
    if (warp == 0) {
      features_reverse(T, Bl, C.XB, GC{D.sbar_ext + (size_t)i * T.ext_k0p, 1});
      hinge_reverse(T, Bl, C.XB);
    }
    mw_barrier();
  }
  if (t >= 0) {
    mw_reverse_step<Q>(T, D, C, t, D.state, tn >= Tw, warp, bm, jm);
  } else {
    if (warp == 0 && T.loss_kind == 3) loss_initial_reverse(T, D, C);
    mw_barrier();
  }
  for (int f = warp; f < nf; f += 4) D.grad_state0[(size_t)f * Bp + i] = C.XB[f];
}

// Wide controller, reverse mode one step per launch. Launch t adds the adjoint of the input
// features s_{t+1} (from the products of step t+1, DevPtrs.sbar_ext) to the state adjoint of
// x_{t+1}, then reverses step t down to the controller-output adjoint (DevPtrs.ub_ext). The state
// adjoint is carried between launches in grad_state0 (zeroed before the first). Launch t = -1
// adds the adjoint of s_0 and the initial term of the loss.
template <class Q>
__global__ void __launch_bounds__(32, 1) k_backward_ext(const __grid_constant__ DevTopo T, const __grid_constant__ DevPtrs D,
                                                        int t) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  const int Bp = T.Bp;
  const int nf = 18 * T.nb;
  float* sm = g_smem + lane;
  BwdCtx C{SL{sm}, SL{sm + T.sm_x * 32}, SL{sm + T.sm_xb * 32}, SL{sm + T.sm_vb * 32}, SL{sm + T.sm_rc * 32},
           SL{sm + T.sm_sbar * 32}, GC{D.prm + i, Bp}, GL{D.grad_prm + i, Bp}, i, D.dloss[i]};
  const int Tw = warp_horizon(D, i);
  if (t >= Tw) return;  // this warp's rollout ended before step t
  const size_t sbytes = (size_t)nf * Bp;
  for (int f = 0; f < nf; ++f) C.XB[f] = D.grad_state0[(size_t)f * Bp + i];
  const int tn = t + 1;
  if (tn < Tw) {  // adjoint of the features of x_{t+1}
    copy_state_to_smem(T, D.ckpt + (size_t)tn * sbytes, i, C.X);
    LaneT<GSR> L{C.S, C.P, GSR{D.ckpt}, i};
    BLaneT<GSR> Bl{L, C.X, C.G, GC{D.ckpt, 32}};
    hinge_kinematics(T, L, C.X);
    for (int j = 0; j < T.nj; ++j) {
      C.S[T.sm_thb + j] = 0.f; C.S[T.sm_thdb + j] = 0.f; C.S[T.sm_wstb + j] = 0.f;
      C.S.s3(T.sm_uab + 3 * j, f3(0.f, 0.f, 0.f));
    }
    features_reverse(T, Bl, C.XB, GC{D.sbar_ext + (size_t)i * T.ext_k0p, 1});
    hinge_reverse(T, Bl, C.XB);
  }
  if (t >= 0) {
    reverse_step<Q, GSR>(T, D, C, t, t, D.ckpt + (size_t)t * sbytes, tn < Tw ? D.ckpt + (size_t)tn * sbytes : D.state);
  } else if (T.loss_kind == 3) {
    loss_initial_reverse(T, D, C);
  }
  for (int f = 0; f < nf; ++f) D.grad_state0[(size_t)f * Bp + i] = C.XB[f];
}

// Per-instance gradient check after a reverse pass: status bit DPK_ST_NAN_GRAD set where the
// state or parameter adjoint holds a non-finite value, cleared elsewhere.
