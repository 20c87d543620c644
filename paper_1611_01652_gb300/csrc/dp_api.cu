// Host implementation of the C ABI declared in include/dp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dp.h"
#include "dp_kernels.h"
#include "dp_mma.cuh"
#include "dp_world.h"

namespace {

thread_local std::string g_err = "no error";

dp_status fail(dp_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(DP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t round32(size_t x) { return (x + 31) / 32 * 32; }

}  // namespace


namespace {

template <class T>
dp_status dalloc(dp_world* w, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DP_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  w->allocs.push_back(*p);
  return DP_OK;
}

#define TRY(x)                  \
  do {                          \
    dp_status s_ = (x);         \
    if (s_ != DP_OK) return s_; \
  } while (0)

struct Slot {
  int kind, idx, sub, a, b, normal;
};

// Canonical slot order: joints (3 linear + 2 angular rows per hinge), limits, motors, ground
// contacts (normal, 2 friction per sphere), pair contacts.
std::vector<Slot> build_slots(const dp_batch_desc* d) {
  std::vector<Slot> s;
  for (int j = 0; j < d->n_joints; ++j) {
    int a = d->joint_body[2 * j], b = d->joint_body[2 * j + 1];
    for (int k = 0; k < 3; ++k) s.push_back({RK_JLIN, j, k, a, b, -1});
    if (d->joint_type[j] == DP_JOINT_HINGE)
      for (int k = 0; k < 2; ++k) s.push_back({RK_JANG, j, k, a, b, -1});
  }
  for (int j = 0; j < d->n_joints; ++j)
    if (d->joint_type[j] == DP_JOINT_HINGE && (d->joint_flags[j] & DP_FLAG_LIMIT))
      s.push_back({RK_LIMIT, j, 0, d->joint_body[2 * j], d->joint_body[2 * j + 1], -1});
  for (int j = 0; j < d->n_joints; ++j)
    if (d->joint_type[j] == DP_JOINT_HINGE && (d->joint_flags[j] & DP_FLAG_MOTOR))
      s.push_back({RK_MOTOR, j, 0, d->joint_body[2 * j], d->joint_body[2 * j + 1], -1});
  for (int q = 0; q < d->n_spheres; ++q) {
    int n = (int)s.size(), a = d->sphere_body[q];
    s.push_back({RK_GN, q, 0, a, -1, -1});
    s.push_back({RK_GT, q, 0, a, -1, n});
    s.push_back({RK_GT, q, 1, a, -1, n});
  }
  for (int q = 0; q < d->n_pairs; ++q) {
    int n = (int)s.size();
    int a = d->sphere_body[d->pair_sphere[2 * q]], b = d->sphere_body[d->pair_sphere[2 * q + 1]];
    s.push_back({RK_PN, q, 0, a, b, -1});
    s.push_back({RK_PT, q, 0, a, b, n});
    s.push_back({RK_PT, q, 1, a, b, n});
  }
  return s;
}

dp_status validate(const dp_batch_desc* d) {
  if (!d) return fail(DP_EINVAL, "descriptor is NULL");
  if (d->n_instances < 1) return fail(DP_EINVAL, "n_instances must be >= 1");
  if (d->n_bodies < 1 || d->n_bodies > DP_MAX_BODIES) return fail(DP_EINVAL, "n_bodies out of range [1, 32]");
  if (d->n_joints < 0 || d->n_joints > DP_MAX_JOINTS) return fail(DP_EINVAL, "n_joints out of range [0, 32]");
  if (d->n_spheres < 0 || d->n_spheres > DP_MAX_SPHERES) return fail(DP_EINVAL, "n_spheres out of range [0, 32]");
  if (d->n_pairs < 0 || d->n_pairs > DP_MAX_PAIRS) return fail(DP_EINVAL, "n_pairs out of range [0, 32]");
  if (d->horizon < 1) return fail(DP_EINVAL, "horizon must be >= 1");
  if (d->horizons)
    for (int i = 0; i < d->n_instances; ++i)
      if (d->horizons[i] < 1 || d->horizons[i] > d->horizon)
        return fail(DP_EINVAL, "horizons[" + std::to_string(i) + "] out of range [1, horizon]");
  if (d->dw_splits < 0) return fail(DP_EINVAL, "dw_splits must be >= 0");
  if (!(d->grad_decay >= 0.f && d->grad_decay <= 1.f)) return fail(DP_EINVAL, "grad_decay must lie in [0, 1]");
  if (d->n_recurrent < 0 || d->n_recurrent > 64) return fail(DP_EINVAL, "n_recurrent out of range [0, 64]");
  if (d->iters < 1) return fail(DP_EINVAL, "iters must be >= 1");
  if (!(d->dt > 0.f)) return fail(DP_EINVAL, "dt must be > 0");
  if (d->ckpt_every < 0) return fail(DP_EINVAL, "ckpt_every must be >= 0");
  if (!d->mass || !d->inertia || !d->state0) return fail(DP_EINVAL, "mass, inertia and state0 are required");
  if (d->n_joints > 0 && (!d->joint_type || !d->joint_body || !d->joint_flags || !d->anchor || !d->axis || !d->ref ||
                          !d->limit || !d->motor))
    return fail(DP_EINVAL, "joint arrays are required when n_joints > 0");
  if (d->n_spheres > 0 && (!d->sphere_body || !d->sph_off || !d->sph_rad || !d->sph_mu || !d->sph_e))
    return fail(DP_EINVAL, "sphere arrays are required when n_spheres > 0");
  if (d->n_pairs > 0 && !d->pair_sphere) return fail(DP_EINVAL, "pair_sphere is required when n_pairs > 0");
  for (int j = 0; j < d->n_joints; ++j) {
    int a = d->joint_body[2 * j], b = d->joint_body[2 * j + 1];
    if (b < 0 || b >= d->n_bodies || a < -1 || a >= d->n_bodies || a == b)
      return fail(DP_EINVAL, "joint " + std::to_string(j) + ": bad bodies");
    if (d->joint_type[j] != DP_JOINT_BALL && d->joint_type[j] != DP_JOINT_HINGE)
      return fail(DP_EINVAL, "joint " + std::to_string(j) + ": bad type");
    if (d->joint_type[j] == DP_JOINT_BALL && d->joint_flags[j] != 0)
      return fail(DP_EINVAL, "joint " + std::to_string(j) + ": limits/motors need a hinge");
  }
  for (int q = 0; q < d->n_spheres; ++q)
    if (d->sphere_body[q] < 0 || d->sphere_body[q] >= d->n_bodies) return fail(DP_EINVAL, "sphere body out of range");
  for (int q = 0; q < d->n_pairs; ++q) {
    int k = d->pair_sphere[2 * q], l = d->pair_sphere[2 * q + 1];
    if (k < 0 || l < 0 || k >= d->n_spheres || l >= d->n_spheres || d->sphere_body[k] == d->sphere_body[l])
      return fail(DP_EINVAL, "pair " + std::to_string(q) + ": spheres must exist and sit on different bodies");
  }
  if (d->loss_body < 0 || d->loss_body >= d->n_bodies) return fail(DP_EINVAL, "loss_body out of range");
  if (d->loss_kind < 0 || d->loss_kind > 3 || d->loss_mode < 0 || d->loss_mode > 1)
    return fail(DP_EINVAL, "bad loss kind/mode");
  if (d->n_layers < 0 || d->n_layers > DP_MAX_LAYERS) return fail(DP_EINVAL, "n_layers out of range [0, 6]");
  for (int l = 0; l <= d->n_layers && d->n_layers > 0; ++l)
    if (d->widths[l] < 1 || d->widths[l] > 4096) return fail(DP_EINVAL, "controller width out of range");
  if (d->n_layers > 0 && (d->imu_body < 0 || d->imu_body >= d->n_bodies)) return fail(DP_EINVAL, "imu_body out of range");
  for (int i = 0; i < d->n_instances; ++i)
    for (int b = 0; b < d->n_bodies; ++b) {
      if (!(d->mass[i * d->n_bodies + b] > 0.f)) return fail(DP_EINVAL, "masses must be > 0");
      for (int k = 0; k < 3; ++k)
        if (!(d->inertia[(i * d->n_bodies + b) * 3 + k] > 0.f)) return fail(DP_EINVAL, "inertias must be > 0");
    }
  for (int i = 0; i < d->n_instances; ++i)
    for (int j = 0; j < d->n_joints; ++j)
      if (d->joint_type[j] == DP_JOINT_HINGE && (d->joint_flags[j] & DP_FLAG_LIMIT) &&
          !(d->limit[(i * d->n_joints + j) * 2] < d->limit[(i * d->n_joints + j) * 2 + 1]))
        return fail(DP_EINVAL, "joint limits need lower < upper");
  return DP_OK;
}

int feature_count(const dp_batch_desc* d, int n_motors) {
  int n = 0;
  if (d->features & DP_F_ANGLES) n += n_motors;
  if (d->features & DP_F_RATES) n += n_motors;
  if (d->features & DP_F_CLOCK) n += 2;
  if (d->features & DP_F_IMU) n += 6;
  if (d->features & DP_F_TARGET) n += 3;
  return n;
}

// Shared-memory plan (units of 32 floats per warp). Forward kernel: controller activations on
// chip; backward kernel: row-adjoint accumulators on chip, activations in the global dump.
void plan_smem(DevTopo& T, bool backward, int smem_floats_max, bool rows_on_chip = true) {
  int o = 0;
  auto take = [&](int n) { int r = o; o += std::max(n, 1); return r; };
  T.sm_x = take(18 * T.nb);
  T.sm_iinv = take(6 * T.nb);
  T.sm_invm = take(T.nb);
  T.sm_th = take(T.nj);
  T.sm_thd = take(T.nj);
  T.sm_ua = take(3 * T.nj);
  T.sm_wst = take(T.nj);
  T.sm_wbr = take(T.nj);
  T.sm_lam = take(T.nslots);
  T.sm_h = take(T.n_rec);
  // warm-start scratch (features, outputs, harvest row ids): the joint arrays above are dead
  // once the rows are assembled, so they host it when they are large enough
  const int wsneed = 19 + T.n_wsg;
  const int jreg = T.sm_wbr + std::max(T.nj, 1) - T.sm_th;
  T.sm_ws = wsneed <= jreg ? T.sm_th : take(wsneed);
  T.sm_x0 = T.sm_u = 0;
  T.sm_rows = -1;
  if (!backward) {
    // controller activations and constraint rows share one region: the rows are assembled after
    // the servo targets have consumed the controller output
    for (int l = 0; l <= DPK_MAXL; ++l) T.sm_act[l] = 0;
    const int region = o;
    int acts = 0;
    if (T.ext_ctrl) {  // wide controller: only its input features and its output are on chip
      T.sm_act[0] = region;
      T.sm_act[T.n_layers] = region + T.widths[0];
      acts = T.widths[0] + T.widths[T.n_layers];
    } else if (T.n_layers > 0) {
      for (int l = 0; l <= T.n_layers; ++l) { T.sm_act[l] = region + acts; acts += T.widths[l]; }
    } else {
      acts = 1;
    }
    const int rows = T.nslots * RF_N;
    if (rows_on_chip && (region + std::max(acts, rows)) * 32 <= smem_floats_max) {
      T.sm_rows = region;
      o = region + std::max(acts, rows);
    } else {
      o = region + acts;
    }
    T.sm_xb = T.sm_vb = T.sm_thb = T.sm_thdb = T.sm_uab = T.sm_wstb = T.sm_iinvb = T.sm_invmb = T.sm_rc = T.sm_sbar = 0;
    T.sm_vw = T.sm_zb = T.sm_hb = 0;
  } else {
    for (int l = 0; l <= DPK_MAXL; ++l) T.sm_act[l] = 0;
    T.sm_xb = take(18 * T.nb);
    T.sm_vb = take(6 * T.nb);
    T.sm_thb = take(T.nj);
    T.sm_thdb = take(T.nj);
    T.sm_uab = take(3 * T.nj);
    T.sm_wstb = take(T.nj);
    T.sm_iinvb = take(9 * T.nb);
    T.sm_invmb = take(T.nb);
    T.sm_rc = take(12 * T.nslots);
    // the in-step controller's input adjoint (the wide controller's goes to the batched products)
    T.sm_sbar = take(T.n_layers > 0 && !T.ext_ctrl ? T.widths[0] : 1);
    // the run-time reverse sweep's working velocities, or the multi-warp sweep's hand-off ring
    // (compiled topologies: the worlds that run the four-warp kernels)
    const bool mw = T.topo_id != 0;
    T.sm_vw = T.sm_ring = take(mw ? std::max(6 * T.nb, 4 * DPK_MW_CH) : 6 * T.nb);
    T.sm_hb = take(T.n_rec);
    // controller-reverse ping-pong buffers: the row-adjoint region is free by then
    int maxw = 1;
    for (int l = 0; l <= T.n_layers && T.n_layers > 0; ++l)
      if (!T.ext_ctrl || l == 0 || l == T.n_layers) maxw = std::max(maxw, T.widths[l]);
    T.sm_zb = 2 * maxw <= 12 * T.nslots ? T.sm_rc : take(2 * maxw);
  }
  T.sm_total = o;
}

void pack_param(std::vector<float>& h, int Bp, int B, int field0, int n, const float* src) {
  if (!src) return;
  for (int i = 0; i < Bp; ++i) {
    int si = i < B ? i : B - 1;
    for (int f = 0; f < n; ++f) h[(size_t)(field0 + f) * Bp + i] = src[(size_t)si * n + f];
  }
}

}  // namespace

// Error reporting for the other C-ABI translation units of the library.
dp_status dp_internal_fail(dp_status s, const char* msg) { return fail(s, msg); }

extern "C" {

const char* dp_last_error(void) { return g_err.c_str(); }

dp_status dp_create_world(const dp_batch_desc* d, void* stream, dp_world** out) {
  if (!out) return fail(DP_EINVAL, "out is NULL");
  *out = nullptr;
  TRY(validate(d));
  dp_world* w = new dp_world();
  auto cleanup = [&](dp_status s) {
    dp_free(w);
    return s;
  };
  w->stream = (cudaStream_t)stream;
  DevTopo T;
  std::memset(&T, 0, sizeof(T));
  const int B = d->n_instances, Bp = (int)round32(B);
  w->B = B;
  w->Bp = Bp;
  T.B = B;
  T.Bp = Bp;
  T.nb = d->n_bodies;
  T.nj = d->n_joints;
  T.ns = d->n_spheres;
  T.np = d->n_pairs;
  T.iters = d->iters;
  T.horizon = d->horizon;
  T.features = d->features;
  T.imu_body = d->imu_body;
  T.loss_kind = d->loss_kind;
  T.loss_mode = d->loss_mode;
  T.loss_body = d->loss_body;
  T.n_layers = d->n_layers;
  T.skip = d->n_layers > 0 ? d->skip : 0;
  T.ctrl_round = d->ctrl_fp32 ? 0 : 1;
  for (int k = 0; k < 3; ++k) T.gravity[k] = d->gravity[k];
  T.dt = d->dt;
  T.ground_z = d->ground_z;
  T.beta = d->beta;
  T.gamma = d->gamma;
  T.slop = d->slop;
  T.clock_hz = d->clock_hz;
  for (int j = 0; j < T.nj; ++j) {
    T.jtype[j] = (int8_t)d->joint_type[j];
    T.ja[j] = (int8_t)d->joint_body[2 * j];
    T.jb[j] = (int8_t)d->joint_body[2 * j + 1];
    T.jflags[j] = (int8_t)d->joint_flags[j];
    T.jmotor[j] = -1;
  }
  for (int j = 0; j < T.nj; ++j)
    if (d->joint_type[j] == DP_JOINT_HINGE && (d->joint_flags[j] & DP_FLAG_MOTOR)) {
      T.jmotor[j] = (int8_t)T.n_motors;
      T.motor_joint[T.n_motors++] = (int8_t)j;
    }
  for (int q = 0; q < T.ns; ++q) T.sbody[q] = (int8_t)d->sphere_body[q];
  for (int q = 0; q < T.np; ++q) {
    T.pk[q] = (int8_t)d->pair_sphere[2 * q];
    T.pl[q] = (int8_t)d->pair_sphere[2 * q + 1];
  }
  // slots, greedy colouring over non-world bodies, sweep order (colour, slot)
  std::vector<Slot> slots = build_slots(d);
  T.nslots = (int)slots.size();
  if (T.nslots > DPK_MAXSLOT) return cleanup(fail(DP_EINVAL, "too many constraint slots"));
  std::vector<int> col(T.nslots, 0), ord(T.nslots);
  for (int i = 0; i < T.nslots; ++i) {
    std::vector<char> used(T.nslots + 1, 0);
    for (int k = 0; k < i; ++k) {
      bool share = (slots[i].a >= 0 && (slots[i].a == slots[k].a || slots[i].a == slots[k].b)) ||
                   (slots[i].b >= 0 && (slots[i].b == slots[k].a || slots[i].b == slots[k].b));
      if (share) used[col[k]] = 1;
    }
    int c = 0;
    while (used[c]) ++c;
    col[i] = c;
  }
  for (int i = 0; i < T.nslots; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return col[x] < col[y]; });
  for (int s = 0; s < T.nslots; ++s) {
    T.skind[s] = (uint8_t)slots[s].kind;
    T.sidx[s] = (uint8_t)slots[s].idx;
    T.ssub[s] = (uint8_t)slots[s].sub;
    T.sa[s] = (int8_t)slots[s].a;
    T.sb[s] = (int8_t)slots[s].b;
    T.snormal[s] = (int16_t)slots[s].normal;
    T.order[s] = (int16_t)ord[s];
    w->kind[s] = slots[s].kind;
    w->colour[s] = col[s];
  }
  // body ownership of the multi-warp reverse pass (stages outside the sweeps): longest processing
  // time over four warps by the number of row sides touching each body (ties: lower index)
  {
    int cnt[DPK_MAXB] = {0}, load[4] = {0};
    bool done[DPK_MAXB] = {false};
    for (const Slot& q : slots) {
      if (q.a >= 0) ++cnt[q.a];
      if (q.b >= 0) ++cnt[q.b];
    }
    for (int k = 0; k < T.nb; ++k) {
      int best = -1;
      for (int b = 0; b < T.nb; ++b)
        if (!done[b] && (best < 0 || cnt[b] > cnt[best])) best = b;
      done[best] = true;
      int h = 0;
      for (int g = 1; g < 4; ++g)
        if (load[g] < load[h]) h = g;
      T.mw_own[best] = (int8_t)h;
      load[h] += cnt[best];
    }
    for (int g = 0; g < 4; ++g) T.mw_bmask[g] = T.mw_jmask[g] = 0u;
    for (int b = 0; b < T.nb; ++b) T.mw_bmask[T.mw_own[b]] |= 1u << b;
    for (int j = 0; j < T.nj; ++j) T.mw_jmask[T.mw_own[T.jb[j]]] |= 1u << j;
    // each warp's slots with an owned side, in slot order, and which sides it owns
    for (int g = 0; g < 4; ++g) {
      int n = 0;
      for (int q = 0; q < T.nslots; ++q) {
        const bool oa = T.sa[q] >= 0 && T.mw_own[T.sa[q]] == g, ob = T.sb[q] >= 0 && T.mw_own[T.sb[q]] == g;
        if (oa || ob) T.mw_slot[g][n++] = (int16_t)(q | (oa ? MW_SLOT_A : 0) | (ob ? MW_SLOT_B : 0));
      }
      T.mw_nslot[g] = (int16_t)n;
    }
  }
  // warm-start groups, in slot order of their first row
  T.n_wsg = 0;
  for (int s = 0; s < T.nslots; ++s) {
    const Slot& q = slots[s];
    int type = -1, g3[3] = {s, s + 1, s + 2};
    if (q.kind == RK_JLIN && q.sub == 0) {
      type = WSG_JOINT;
    } else if (q.kind == RK_JANG && q.sub == 0) {
      type = WSG_HINGE;
      g3[2] = -1;
      for (int k = 0; k < T.nslots; ++k)
        if (slots[k].kind == RK_MOTOR && slots[k].idx == q.idx) g3[2] = k;
    } else if (q.kind == RK_GN) {
      type = WSG_GROUND;
    } else if (q.kind == RK_PN) {
      type = WSG_PAIR;
    }
    if (type < 0) continue;
    T.wsg_type[T.n_wsg] = (int8_t)type;
    for (int k = 0; k < 3; ++k) T.wsg_slot[T.n_wsg][k] = (int16_t)g3[k];
    ++T.n_wsg;
  }
  // parameter fields
  int o = 0;
  T.o_mass = o; o += T.nb;
  T.o_inertia = o; o += 3 * T.nb;
  T.o_anchor = o; o += 6 * T.nj;
  T.o_axis = o; o += 6 * T.nj;
  T.o_ref = o; o += 6 * T.nj;
  T.o_limit = o; o += 2 * T.nj;
  T.o_motor = o; o += 3 * T.nj;
  T.o_sph_off = o; o += 3 * T.ns;
  T.o_sph_rad = o; o += T.ns;
  T.o_sph_mu = o; o += T.ns;
  T.o_sph_e = o; o += T.ns;
  T.o_loss_point = o; o += 3;
  T.o_loss_target = o; o += 3;
  T.n_pfields = o;
  // controller
  int64_t np_ = 0;
  int wtot = 0;
  if (T.n_layers > 0) {
    for (int l = 0; l <= T.n_layers; ++l) T.widths[l] = d->widths[l];
    if (feature_count(d, T.n_motors) + d->n_recurrent > T.widths[0])
      return cleanup(fail(DP_EINVAL, "controller input width is smaller than the selected features (+ recurrent state)"));
    if (d->n_recurrent > 0 && (T.skip || T.n_motors + d->n_recurrent > T.widths[T.n_layers]))
      return cleanup(fail(DP_EINVAL, "a recurrent controller needs no skip layer and widths[n_layers] >= motors + n_recurrent"));
    const int nl = T.n_layers + (T.skip ? 1 : 0);
    for (int l = 0; l < nl; ++l) {
      int ni = l < T.n_layers ? T.widths[l] : T.widths[0];
      int no_ = l < T.n_layers ? T.widths[l + 1] : T.widths[T.n_layers];
      int nop = (no_ + 7) & ~7, nip = (ni + 7) & ~7;
      T.w_off[l] = wtot;
      wtot += std::max(ni * nop, no_ * nip);
      np_ += (int64_t)ni * no_ + no_;
    }
    int r = 0;
    for (int l = 0; l <= T.n_layers; ++l) { T.dump_act[l] = r; r += T.widths[l]; }
    for (int l = 0; l < T.n_layers; ++l) { T.dump_del[l] = r; r += T.widths[l + 1]; }
    T.dump_rows = r;
  }
  T.n_params = (int)np_;
  T.ws = 0;
  T.ws_net = 0;
  T.n_rec = T.n_layers > 0 ? d->n_recurrent : 0;
  T.ws_alpha = 0.7f;
  T.grad_decay = d->grad_decay > 0.f ? d->grad_decay : 1.f;
  // bfloat16 controllers K0-H-H-NO with K0 <= 32, NO <= 16 and H in {64, 128, 256} run on the
  // tensor cores inside the step (recurrent ones too: h is among the inputs and outputs)
  T.mlp_tc = T.n_layers == 3 && !T.skip && T.ctrl_round && T.widths[0] <= CTRL_TC_KP0 && T.widths[3] <= CTRL_TC_NOP &&
             T.widths[1] == T.widths[2] && ctrl_tc_width(T.widths[1]) && !getenv("DP_FORCE_SIMT_CONTROLLER");
  // wide bfloat16 controllers (hidden layers beyond 256) run as batched tensor-core products
  // between step launches; DP_FORCE_WIDE_CONTROLLER selects that path for any eligible network
  {
    const bool shape = T.n_rec == 0 && T.n_layers == 3 && !T.skip && T.ctrl_round && T.widths[1] % 64 == 0 && T.widths[2] % 64 == 0 &&
                       T.widths[3] <= 8 && T.widths[0] <= 256;
    const bool wide = T.n_layers == 3 && (T.widths[1] > 256 || T.widths[2] > 256);
    T.ext_ctrl = shape && (wide || getenv("DP_FORCE_WIDE_CONTROLLER") != nullptr);
    if (T.ext_ctrl) {
      T.mlp_tc = 0;
      T.ext_k0p = (T.widths[0] + 63) / 64 * 64;
      T.ext_nop = 8;
      w->ext.k0p = T.ext_k0p;
      w->ext.h1 = T.widths[1];
      w->ext.h2 = T.widths[2];
      w->ext.no = T.widths[3];
      size_t o = 0;
      w->ext.w1 = o; o += (size_t)T.widths[1] * T.ext_k0p;
      w->ext.w2 = o; o += (size_t)T.widths[2] * T.widths[1];
      w->ext.w3 = o; o += (size_t)8 * T.widths[2];
      w->ext.w3t = o; o += (size_t)T.widths[2] * 16;
      w->ext.w2t = o; o += (size_t)T.widths[1] * T.widths[2];
      w->ext.w1t = o; o += (size_t)T.ext_k0p * T.widths[1];
      w->ext.size = o;
    }
  }
  T.topo_id = match_compiled_topology(T, T.nb, T.nj, T.ns, T.np, d->joint_type, d->joint_body, d->joint_flags,
                                      d->sphere_body, d->pair_sphere);
  if (getenv("DP_FORCE_RUNTIME_TOPOLOGY")) T.topo_id = 0;
  T.one_warp = d->one_warp ? 1 : 0;
  // a compiled topology's kernels carry one width of the tensor-core controller: another width
  // runs on the SIMT path
  if (T.topo_id != 0 && T.widths[1] != compiled_ctrl_width(T.topo_id)) T.mlp_tc = 0;
  w->n_params = np_;
  w->w_total = wtot;
  w->Tf = T;
  w->Tb = T;
  int dev = 0, smem_max = 0;
  CU(cudaGetDevice(&dev));
  w->device = dev;
  CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  plan_smem(w->Tf, false, smem_max / (int)sizeof(float), d->rows_global == 0);
  plan_smem(w->Tb, true, smem_max / (int)sizeof(float));
  size_t need = (size_t)std::max(w->Tf.sm_total, w->Tb.sm_total) * 32 * sizeof(float);
  if (need > (size_t)smem_max) {
    dp_status s = fail(DP_EINVAL, "robot too large: needs " + std::to_string(need) + " bytes of shared memory per warp, the device offers " +
                                      std::to_string(smem_max));
    return cleanup(s);
  }
  // Memory plan. With enough device memory the rollout records every step's solver tape and the
  // backward pass only reads it (no recomputation). Otherwise states are checkpointed every K
  // steps and the backward pass recomputes one K-step segment at a time with its tape.
  const int nf = 18 * T.nb;
  w->nf = nf;
  const size_t state_bytes = (size_t)nf * Bp * sizeof(float);
  // tape record of one (step, warp): rows, impulses, per-sweep velocities, post-impulse
  // velocities, clamp branches; 32 lanes interleaved; 16-byte multiple for bulk prefetches
  {
    long long o = (long long)T.nslots * RF_N * 32 * 4;
    T.rec_lam = o;
    o += (long long)T.iters * T.nslots * 32 * 4;
    T.rec_viter = o;
    o += (long long)T.iters * T.nb * 6 * 32 * 4;
    T.rec_vminus = o;
    o += (long long)T.nb * 6 * 32 * 4;
    T.rec_br = o;
    o += (long long)T.iters * T.nslots * 32;
    o = (o + 15) / 16 * 16;
    T.rec_lam0 = o;
    if (d->warmstart) o += (long long)T.nslots * 32 * 4;
    T.rec_bytes = (o + 255) / 256 * 256;
    for (DevTopo* t2 : {&w->Tf, &w->Tb}) {
      t2->rec_lam = T.rec_lam;
      t2->rec_viter = T.rec_viter;
      t2->rec_vminus = T.rec_vminus;
      t2->rec_br = T.rec_br;
      t2->rec_lam0 = T.rec_lam0;
      t2->rec_bytes = T.rec_bytes;
    }
  }
  const size_t tape_step_bytes = (size_t)T.rec_bytes * (Bp / 32);
  const size_t dump_bytes = (size_t)T.dump_rows * T.horizon * Bp * sizeof(float);
  size_t free_b = 0, total_b = 0;
  CU(cudaMemGetInfo(&free_b, &total_b));
  const size_t fixed = (size_t)T.nslots * RF_N * Bp * sizeof(float) + 8 * state_bytes + ((size_t)64 << 20);
  const size_t usable = (size_t)(0.85 * (double)free_b);
  const size_t budget = usable > dump_bytes + fixed ? usable - dump_bytes - fixed : 0;
  int K = d->ckpt_every;
  bool full = false;
  auto seg_bytes = [&](int k) {
    return (size_t)((T.horizon + k - 1) / k) * state_bytes + (size_t)k * tape_step_bytes + (size_t)(k + 1) * state_bytes;
  };
  if (K == 0) {
    if ((size_t)T.horizon * (tape_step_bytes + state_bytes) <= budget) {
      full = true;
      K = 1;
    } else {
      int best = 1;
      for (int k = 1; k <= T.horizon; ++k)
        if (seg_bytes(k) < seg_bytes(best)) best = k;
      if (seg_bytes(best) > budget)
        return cleanup(fail(DP_ENOMEM, "not enough device memory for checkpoints and one segment's tape"));
      K = best;
    }
  }
  K = std::min(K, T.horizon);
  if (T.ext_ctrl && !full)
    return cleanup(fail(DP_ENOMEM, "a wide controller needs the whole solver tape in device memory"));
  const int n_ckpt = (T.horizon + K - 1) / K;
  const int tape_steps = full ? T.horizon : K;
  DevPtrs& D = w->D;
  std::memset(&D, 0, sizeof(D));
  D.ckpt_every = K;
  D.n_ckpt = n_ckpt;
  D.tape_steps = tape_steps;
  D.tape_full = full ? 1 : 0;
  // device buffers
  float* prm = nullptr;
  if (dalloc(w, &prm, (size_t)T.n_pfields * Bp)) return cleanup(DP_ENOMEM);
  D.prm = prm;
  const size_t Bz = (size_t)Bp;
  if (dalloc(w, &D.state, (size_t)nf * Bz) || dalloc(w, &w->x0, (size_t)nf * Bz) ||
      dalloc(w, &D.ckpt, (size_t)n_ckpt * nf * Bz) || dalloc(w, &D.seg, full ? (size_t)1 : (size_t)(K + 1) * nf * Bz) ||
      dalloc(w, &D.rows, (size_t)T.nslots * RF_N * Bz) ||
      dalloc(w, &D.tape, (size_t)tape_steps * tape_step_bytes) || dalloc(w, &D.loss, Bz) || dalloc(w, &D.dloss, Bz) ||
      dalloc(w, &D.grad_prm, (size_t)T.n_pfields * Bz) || dalloc(w, &D.grad_state0, (size_t)nf * Bz) ||
      dalloc(w, &D.status, Bz))
    return cleanup(DP_ENOMEM);
  if (T.n_layers > 0) {
    if (dalloc(w, &D.dump, (size_t)T.dump_rows * T.horizon * Bp) || dalloc(w, &w->Wmaster, (size_t)np_) ||
        dalloc(w, &w->Wt, (size_t)wtot) || dalloc(w, &w->Wn, (size_t)wtot) || dalloc(w, &w->Wb, (size_t)wtot) ||
        dalloc(w, &w->dW_stage, (size_t)np_))
      return cleanup(DP_ENOMEM);
    // columns of steps a warp never reaches (uneven horizons) stay zero for the dW reduction
    CU(cudaMemsetAsync(D.dump, 0, sizeof(float) * (size_t)T.dump_rows * T.horizon * Bp, w->stream));
    CU(cudaMemsetAsync(w->Wt, 0, sizeof(float) * wtot, w->stream));
    CU(cudaMemsetAsync(w->Wn, 0, sizeof(float) * wtot, w->stream));
    CU(cudaMemsetAsync(w->Wb, 0, sizeof(float) * wtot, w->stream));
    size_t N = (size_t)T.horizon * Bp;
    w->splits = d->dw_splits > 0 ? std::min(d->dw_splits, 256) : (int)std::min<size_t>(256, (N + 16383) / 16384);
    size_t maxlayer = 0;
    for (int l = 0; l <= T.n_layers; ++l) maxlayer = std::max(maxlayer, (size_t)T.widths[l]);
    // the wide controller's tensor-core weight gradient splits its columns up to 20 ways
    w->partial_floats = (size_t)std::max(w->splits, T.ext_ctrl ? 20 : 1) * maxlayer * maxlayer;
    if (dalloc(w, &w->partial, w->partial_floats)) return cleanup(DP_ENOMEM);
    D.Wt = w->Wt;
    D.Wn = w->Wn;
    D.bias = w->Wb;
    if (T.mlp_tc) {
      void* p = nullptr;
      const size_t n = (size_t)ctrl_tc_layout(T.widths[1], T.widths[2]).size;
      if (cudaMalloc(&p, sizeof(__nv_bfloat16) * n) != cudaSuccess) return cleanup(DP_ENOMEM);
      w->allocs.push_back(p);
      w->Wtc = (__nv_bfloat16*)p;
    }
    D.Wtc = w->Wtc;
    if (T.ext_ctrl) {
      const size_t k0p = (size_t)T.ext_k0p, h1 = (size_t)T.widths[1], h2 = (size_t)T.widths[2];
      void* p[4] = {nullptr, nullptr, nullptr, nullptr};
      const size_t nbf[4] = {w->ext.size, Bz * k0p, Bz * h1, Bz * h2};
      for (int k = 0; k < 4; ++k) {
        if (cudaMalloc(&p[k], sizeof(__nv_bfloat16) * nbf[k]) != cudaSuccess) return cleanup(DP_ENOMEM);
        w->allocs.push_back(p[k]);
      }
      w->ext_w = (__nv_bfloat16*)p[0];
      D.s_ext = (__nv_bfloat16*)p[1];
      w->ext_h1 = (__nv_bfloat16*)p[2];
      w->ext_h2 = (__nv_bfloat16*)p[3];
      float* sb = nullptr;
      if (dalloc(w, &D.u_ext, (size_t)T.horizon * Bz * 8) || dalloc(w, &D.ub_ext, Bz * 16) || dalloc(w, &sb, Bz * k0p) ||
          dalloc(w, &w->ext_d1, Bz * h1) || dalloc(w, &w->ext_d2, Bz * h2))
        return cleanup(DP_ENOMEM);
      D.sbar_ext = sb;
    }
  } else {
    float* dummy = nullptr;
    if (dalloc(w, &dummy, 8)) return cleanup(DP_ENOMEM);
    CU(cudaMemsetAsync(dummy, 0, 8 * sizeof(float), w->stream));
    D.Wt = D.Wn = D.bias = dummy;
    D.dump = dummy;
  }
  // warm start (enabled later by dp_set_warmstart), residual sums, harvest counter
  w->ws_capable = d->warmstart != 0;
  if (w->ws_capable) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(__nv_bfloat16) * WsTC::SIZE) != cudaSuccess) return cleanup(DP_ENOMEM);
    w->allocs.push_back(p);
    w->ws_tc = (__nv_bfloat16*)p;
    if (dalloc(w, &w->ws_master, (size_t)WsTC::PARAMS) || dalloc(w, &w->ws_b, (size_t)WsTC::BSIZE))
      return cleanup(DP_ENOMEM);
  }
  int* hz = nullptr;
  if (dalloc(w, &w->resid, Bz) || dalloc(w, &w->harvest_count, 1) || dalloc(w, &D.lam_prev, (size_t)T.nslots * Bz) ||
      dalloc(w, &hz, Bz))
    return cleanup(DP_ENOMEM);
  {
    std::vector<int> hh(Bp);
    for (int i = 0; i < Bp; ++i) hh[i] = d->horizons ? d->horizons[i < B ? i : B - 1] : d->horizon;
    CU(cudaMemcpyAsync(hz, hh.data(), sizeof(int) * Bp, cudaMemcpyHostToDevice, w->stream));
    CU(cudaStreamSynchronize(w->stream));
  }
  D.hz = hz;
  CU(cudaMemsetAsync(w->resid, 0, sizeof(float) * Bz, w->stream));
  CU(cudaMemsetAsync(D.lam_prev, 0, sizeof(float) * (size_t)std::max(T.nslots, 1) * Bz, w->stream));
  D.ckpt_lam = nullptr;
  if (w->ws_capable && !full && dalloc(w, &D.ckpt_lam, (size_t)n_ckpt * T.nslots * Bz)) return cleanup(DP_ENOMEM);
  D.hrec = D.ckpt_h = nullptr;
  if (T.n_rec > 0) {
    if (dalloc(w, &D.hrec, (size_t)T.n_rec * Bz)) return cleanup(DP_ENOMEM);
    CU(cudaMemsetAsync(D.hrec, 0, sizeof(float) * (size_t)T.n_rec * Bz, w->stream));
    if (!full && dalloc(w, &D.ckpt_h, (size_t)n_ckpt * T.n_rec * Bz)) return cleanup(DP_ENOMEM);
  }
  D.ws_tc = w->ws_tc;
  D.ws_b = w->ws_b;
  D.harvest = nullptr;
  D.harvest_count = w->harvest_count;
  D.harvest_max = 0;
  D.u_noise = nullptr;
  D.resid = nullptr;
  const int widest = std::max({nf, 6 * T.nj, 3 * T.nb, 3 * T.ns, T.nslots, 32});
  w->stage_floats = std::max<size_t>((size_t)B * widest, (size_t)np_);
  if (dalloc(w, &w->stage, w->stage_floats)) return cleanup(DP_ENOMEM);
  CU(cudaMemsetAsync(D.status, 0, sizeof(int) * Bp, w->stream));
  // parameters (host pack, one upload)
  std::vector<float> h((size_t)T.n_pfields * Bp, 0.f);
  pack_param(h, Bp, B, T.o_mass, T.nb, d->mass);
  pack_param(h, Bp, B, T.o_inertia, 3 * T.nb, d->inertia);
  pack_param(h, Bp, B, T.o_anchor, 6 * T.nj, d->anchor);
  pack_param(h, Bp, B, T.o_axis, 6 * T.nj, d->axis);
  pack_param(h, Bp, B, T.o_ref, 6 * T.nj, d->ref);
  pack_param(h, Bp, B, T.o_limit, 2 * T.nj, d->limit);
  pack_param(h, Bp, B, T.o_motor, 3 * T.nj, d->motor);
  pack_param(h, Bp, B, T.o_sph_off, 3 * T.ns, d->sph_off);
  pack_param(h, Bp, B, T.o_sph_rad, T.ns, d->sph_rad);
  pack_param(h, Bp, B, T.o_sph_mu, T.ns, d->sph_mu);
  pack_param(h, Bp, B, T.o_sph_e, T.ns, d->sph_e);
  pack_param(h, Bp, B, T.o_loss_point, 3, d->loss_point);
  pack_param(h, Bp, B, T.o_loss_target, 3, d->loss_target);
  CU(cudaMemcpyAsync(prm, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, w->stream));
  std::vector<float> hs((size_t)nf * Bp);
  pack_param(hs, Bp, B, 0, nf, d->state0);
  CU(cudaMemcpyAsync(w->x0, hs.data(), hs.size() * sizeof(float), cudaMemcpyHostToDevice, w->stream));
  CU(cudaMemcpyAsync(D.state, hs.data(), hs.size() * sizeof(float), cudaMemcpyHostToDevice, w->stream));
  CU(cudaStreamSynchronize(w->stream));
  *out = w;
  return DP_OK;
}

void dp_free(dp_world* w) {
  if (!w) return;
  if (w->stream) cudaStreamSynchronize(w->stream);
  else cudaDeviceSynchronize();
  for (void* p : w->allocs) cudaFree(p);
  delete w;
}

int64_t dp_num_params(const dp_world* w) { return w ? w->n_params : -1; }
int32_t dp_num_slots(const dp_world* w) { return w ? w->Tf.nslots : -1; }
int32_t dp_ckpt_every(const dp_world* w) { return w ? w->D.ckpt_every : -1; }
int32_t dp_controller_kind(const dp_world* w) {
  if (!w) return -1;
  const DevTopo& T = w->Tf;
  if (T.n_layers == 0) return DP_CTRL_NONE;
  if (T.ext_ctrl) return DP_CTRL_WIDE;
  return T.mlp_tc ? DP_CTRL_TENSOR : DP_CTRL_SIMT;
}

dp_status dp_schedule(const dp_world* w, int32_t* kind, int32_t* idx, int32_t* sub, int32_t* body_a, int32_t* body_b,
                      int32_t* colour, int32_t* order) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  const DevTopo& T = w->Tf;
  for (int s = 0; s < T.nslots; ++s) {
    if (kind) kind[s] = T.skind[s];
    if (idx) idx[s] = T.sidx[s];
    if (sub) sub[s] = T.ssub[s];
    if (body_a) body_a[s] = T.sa[s];
    if (body_b) body_b[s] = T.sb[s];
    if (colour) colour[s] = w->colour[s];
    if (order) order[s] = T.order[s];
  }
  return DP_OK;
}

static dp_status stage_state_in(dp_world* w, const float* state, float* dst) {
  if (!state) return fail(DP_EINVAL, "state is NULL");
  CU(cudaMemcpyAsync(w->stage, state, sizeof(float) * (size_t)w->B * w->nf, cudaMemcpyDefault, w->stream));
  CU(launch_state_in(w->B, w->Bp, w->nf, w->stage, dst, w->stream));
  return DP_OK;
}

dp_status dp_set_initial_state(dp_world* w, const float* state) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  return stage_state_in(w, state, w->x0);
}

dp_status dp_set_state(dp_world* w, const float* state, int32_t t) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  if (t < 0) return fail(DP_EINVAL, "t must be >= 0");
  TRY(stage_state_in(w, state, w->D.state));
  // the previous impulses belonged to another trajectory: the next step starts without them
  CU(cudaMemsetAsync(w->D.lam_prev, 0, sizeof(float) * (size_t)std::max(w->Tf.nslots, 1) * w->Bp, w->stream));
  if (w->D.hrec) CU(cudaMemsetAsync(w->D.hrec, 0, sizeof(float) * (size_t)w->Tf.n_rec * w->Bp, w->stream));
  w->t_now = t;
  w->have_rollout = false;
  return DP_OK;
}

dp_status dp_get_state(dp_world* w, float* state) {
  if (!w || !state) return fail(DP_EINVAL, "world or state is NULL");
  CU(launch_state_out(w->B, w->Bp, w->nf, w->D.state, w->stage, w->stream));
  CU(cudaMemcpyAsync(state, w->stage, sizeof(float) * (size_t)w->B * w->nf, cudaMemcpyDefault, w->stream));
  return DP_OK;
}

static dp_status stage_weights(dp_world* w, const float* W) {
  if (w->n_params == 0) return DP_OK;
  if (!W) return fail(DP_EINVAL, "the world has a controller: W is required");
  CU(cudaMemcpyAsync(w->Wmaster, W, sizeof(float) * w->n_params, cudaMemcpyDefault, w->stream));
  CU(launch_prep_weights(w->Tf, w->Wmaster, w->Wt, w->Wn, w->Wb, w->stream));
  if (w->Tf.mlp_tc) CU(launch_prep_weights_tc(w->Tf, w->Wmaster, w->Wtc, w->stream));
  if (w->Tf.ext_ctrl) CU(launch_prep_ext(w->ext, w->Tf.widths[0], w->Wmaster, w->ext_w, w->stream));
  return DP_OK;
}

dp_status dp_step(dp_world* w, int32_t n_steps, const float* W, uint8_t* active) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  if (n_steps < 0) return fail(DP_EINVAL, "n_steps must be >= 0");
  if (n_steps == 0) return DP_OK;
  if (w->Tf.ext_ctrl && w->t_now + n_steps > w->Tf.horizon)
    return fail(DP_EINVAL, "with a wide controller dp_step cannot go past the horizon");
  TRY(stage_weights(w, W));
  DevPtrs D = w->D;
  D.active = active;
  D.traj = nullptr;
  if (w->resid_on) {
    D.resid = w->resid;
    w->resid_steps += n_steps;
  }
  if (w->Tf.ext_ctrl)
    CU(ext_forward(w, w->Tf, D, w->t_now, n_steps, 0, 0));
  else
    CU(launch_forward(w->Tf, D, w->x0, w->t_now, n_steps, 0, 0, w->stream));
  w->t_now += n_steps;
  w->have_rollout = false;
  return DP_OK;
}

dp_status dp_rollout(dp_world* w, const float* W, float* loss, float* traj, uint8_t* active) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  TRY(stage_weights(w, W));
  DevPtrs D = w->D;
  D.active = active;
  D.traj = traj;
  if (w->resid_on) {
    D.resid = w->resid;
    w->resid_steps = w->Tf.horizon;
    CU(cudaMemsetAsync(w->resid, 0, sizeof(float) * w->Bp, w->stream));
  }
  CU(cudaMemsetAsync(D.status, 0, sizeof(int) * w->Bp, w->stream));
  if (w->Tf.ext_ctrl)
    CU(ext_forward(w, w->Tf, D, 0, w->Tf.horizon, 1, D.tape_full));
  else
    CU(launch_forward(w->Tf, D, w->x0, 0, w->Tf.horizon, 1, D.tape_full, w->stream));
  if (loss) CU(cudaMemcpyAsync(loss, D.loss, sizeof(float) * w->B, cudaMemcpyDefault, w->stream));
  w->t_now = w->Tf.horizon;
  w->have_rollout = true;
  return DP_OK;
}

dp_status dp_set_warmstart(dp_world* w, const float* W, float alpha) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  if (!w->ws_capable) return fail(DP_EINVAL, "the world was created without warm-start support (desc.warmstart = 0)");
  if (!(alpha >= 0.f && alpha <= 1.f)) return fail(DP_EINVAL, "alpha must lie in [0, 1]");
  if (w->have_rollout) w->have_rollout = false;  // the recorded tape belongs to the other solver
  w->Tf.ws_alpha = w->Tb.ws_alpha = alpha;
  if (!W) {
    w->Tf.ws = w->Tb.ws = 0;
    return DP_OK;
  }
  CU(cudaMemcpyAsync(w->ws_master, W, sizeof(float) * WsTC::PARAMS, cudaMemcpyDefault, w->stream));
  CU(launch_ws_prep(w->ws_master, w->ws_tc, w->ws_b, w->stream));
  w->Tf.ws = w->Tb.ws = 1;
  {  // an identically zero network is the damped start: the kernels skip its evaluation
    std::vector<float> hw(WsTC::PARAMS);
    CU(cudaMemcpyAsync(hw.data(), w->ws_master, sizeof(float) * WsTC::PARAMS, cudaMemcpyDeviceToHost, w->stream));
    CU(cudaStreamSynchronize(w->stream));
    int nz = 0;
    for (float x : hw) nz |= x != 0.f;
    w->Tf.ws_net = w->Tb.ws_net = nz;
  }
  return DP_OK;
}

dp_status dp_set_impulses(dp_world* w, const float* lam) {
  if (!w || !lam) return fail(DP_EINVAL, "world or lam is NULL");
  const int ns = w->Tf.nslots;
  if (ns == 0) return DP_OK;
  CU(cudaMemcpyAsync(w->stage, lam, sizeof(float) * (size_t)w->B * ns, cudaMemcpyDefault, w->stream));
  CU(launch_state_in(w->B, w->Bp, ns, w->stage, w->D.lam_prev, w->stream));
  return DP_OK;
}

dp_status dp_get_impulses(dp_world* w, float* lam) {
  if (!w || !lam) return fail(DP_EINVAL, "world or lam is NULL");
  const int ns = w->Tf.nslots;
  if (ns == 0) return DP_OK;
  CU(launch_state_out(w->B, w->Bp, ns, w->D.lam_prev, w->stage, w->stream));
  CU(cudaMemcpyAsync(lam, w->stage, sizeof(float) * (size_t)w->B * ns, cudaMemcpyDefault, w->stream));
  return DP_OK;
}

dp_status dp_set_params(dp_world* w, const dp_param_grads* p) {
  if (!w || !p) return fail(DP_EINVAL, "world or p is NULL");
  const DevTopo& T = w->Tf;
  struct G { const float* src; int off, n; } groups[] = {
      {p->mass, T.o_mass, T.nb},           {p->inertia, T.o_inertia, 3 * T.nb},  {p->anchor, T.o_anchor, 6 * T.nj},
      {p->limit, T.o_limit, 2 * T.nj},     {p->motor, T.o_motor, 3 * T.nj},      {p->sph_off, T.o_sph_off, 3 * T.ns},
      {p->sph_rad, T.o_sph_rad, T.ns},     {p->sph_mu, T.o_sph_mu, T.ns},        {p->sph_e, T.o_sph_e, T.ns},
      {p->loss_point, T.o_loss_point, 3},  {p->loss_target, T.o_loss_target, 3}};
  for (const G& g : groups) {
    if (!g.src || g.n == 0) continue;
    if ((size_t)w->B * g.n > w->stage_floats) return fail(DP_EINVAL, "staging buffer too small");
    CU(cudaMemcpyAsync(w->stage, g.src, sizeof(float) * (size_t)w->B * g.n, cudaMemcpyDefault, w->stream));
    CU(launch_param_in(w->B, w->Bp, g.off, g.n, w->stage, const_cast<float*>(w->D.prm), w->stream));
  }
  w->have_rollout = false;  // a recorded rollout belongs to the old parameters
  return DP_OK;
}

dp_status dp_set_recurrent(dp_world* w, const float* h) {
  if (!w || !h) return fail(DP_EINVAL, "world or h is NULL");
  const int H = w->Tf.n_rec;
  if (H == 0) return fail(DP_EINVAL, "the world has no recurrent controller state");
  if ((size_t)w->B * H > w->stage_floats) return fail(DP_EINVAL, "staging buffer too small");
  CU(cudaMemcpyAsync(w->stage, h, sizeof(float) * (size_t)w->B * H, cudaMemcpyDefault, w->stream));
  CU(launch_state_in(w->B, w->Bp, H, w->stage, w->D.hrec, w->stream));
  return DP_OK;
}

dp_status dp_get_recurrent(dp_world* w, float* h) {
  if (!w || !h) return fail(DP_EINVAL, "world or h is NULL");
  const int H = w->Tf.n_rec;
  if (H == 0) return fail(DP_EINVAL, "the world has no recurrent controller state");
  if ((size_t)w->B * H > w->stage_floats) return fail(DP_EINVAL, "staging buffer too small");
  CU(launch_state_out(w->B, w->Bp, H, w->D.hrec, w->stage, w->stream));
  CU(cudaMemcpyAsync(h, w->stage, sizeof(float) * (size_t)w->B * H, cudaMemcpyDefault, w->stream));
  return DP_OK;
}

dp_status dp_harvest(dp_world* w, const float* W, const float* u_noise, float* rows, int64_t max_rows,
                     int64_t* n_rows) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  if (!rows || max_rows < 0 || !n_rows) return fail(DP_EINVAL, "rows or n_rows is NULL, or max_rows < 0");
  TRY(stage_weights(w, W));
  DevPtrs D = w->D;
  D.active = nullptr;
  D.traj = nullptr;
  D.harvest = rows;
  D.harvest_max = max_rows;
  D.u_noise = u_noise;
  const DevTopo& T = w->Tf;
  CU(cudaMemsetAsync(w->harvest_count, 0, sizeof(unsigned long long), w->stream));
  CU(cudaMemsetAsync(D.status, 0, sizeof(int) * w->Bp, w->stream));
  if (T.ext_ctrl)
    CU(ext_forward(w, T, D, 0, T.horizon, 1, 0));
  else
    CU(launch_forward(T, D, w->x0, 0, T.horizon, 1, 0, w->stream));
  unsigned long long cnt = 0;
  CU(cudaMemcpyAsync(&cnt, w->harvest_count, sizeof(cnt), cudaMemcpyDeviceToHost, w->stream));
  CU(cudaStreamSynchronize(w->stream));
  *n_rows = (int64_t)std::min<unsigned long long>(cnt, (unsigned long long)max_rows);
  w->t_now = T.horizon;
  w->have_rollout = false;
  return DP_OK;
}

dp_status dp_set_residual(dp_world* w, int32_t on) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  w->resid_on = on != 0;
  w->resid_steps = 0;
  CU(cudaMemsetAsync(w->resid, 0, sizeof(float) * w->Bp, w->stream));
  return DP_OK;
}

dp_status dp_get_residual(dp_world* w, float* resid) {
  if (!w || !resid) return fail(DP_EINVAL, "world or resid is NULL");
  const float sc = w->resid_steps > 0 ? 1.f / (float)w->resid_steps : 0.f;
  CU(launch_scale_out(w->B, w->resid, sc, w->stage, w->stream));
  CU(cudaMemcpyAsync(resid, w->stage, sizeof(float) * w->B, cudaMemcpyDefault, w->stream));
  return DP_OK;
}

dp_status dp_backward(dp_world* w, const float* dloss, float* dW, float* dstate0, const dp_param_grads* dp) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  if (!w->have_rollout) return fail(DP_ESTATE, "dp_backward needs a preceding dp_rollout");
  if (!dloss) return fail(DP_EINVAL, "dloss is NULL");
  const DevTopo& T = w->Tb;
  DevPtrs& D = w->D;
  CU(cudaMemcpyAsync(w->stage, dloss, sizeof(float) * w->B, cudaMemcpyDefault, w->stream));
  CU(launch_pad_scalar(w->B, w->Bp, w->stage, D.dloss, w->stream));
  CU(cudaMemsetAsync(D.grad_prm, 0, sizeof(float) * (size_t)T.n_pfields * w->Bp, w->stream));
  if (T.ext_ctrl)
    CU(ext_backward(w, T, D));
  else
    CU(launch_backward(T, D, w->stream));
  CU(launch_check_grads(w->B, w->Bp, w->nf, T.n_pfields, D.grad_state0, D.grad_prm, D.status, w->stream));
  if (dstate0) {
    CU(launch_state_out(w->B, w->Bp, w->nf, D.grad_state0, w->stage, w->stream));
    CU(cudaMemcpyAsync(dstate0, w->stage, sizeof(float) * (size_t)w->B * w->nf, cudaMemcpyDefault, w->stream));
  }
  if (dp) {
    struct G { float* dst; int off, n; } groups[] = {
        {dp->mass, T.o_mass, T.nb},           {dp->inertia, T.o_inertia, 3 * T.nb},  {dp->anchor, T.o_anchor, 6 * T.nj},
        {dp->limit, T.o_limit, 2 * T.nj},     {dp->motor, T.o_motor, 3 * T.nj},      {dp->sph_off, T.o_sph_off, 3 * T.ns},
        {dp->sph_rad, T.o_sph_rad, T.ns},     {dp->sph_mu, T.o_sph_mu, T.ns},        {dp->sph_e, T.o_sph_e, T.ns},
        {dp->loss_point, T.o_loss_point, 3},  {dp->loss_target, T.o_loss_target, 3}};
    for (const G& g : groups) {
      if (!g.dst || g.n == 0) continue;
      if ((size_t)w->B * g.n > w->stage_floats) return fail(DP_EINVAL, "staging buffer too small");
      CU(launch_param_out(w->B, w->Bp, g.off, g.n, D.grad_prm, w->stage, w->stream));
      CU(cudaMemcpyAsync(g.dst, w->stage, sizeof(float) * (size_t)w->B * g.n, cudaMemcpyDefault, w->stream));
    }
  }
  if (dW && w->n_params > 0 && (T.ext_ctrl || T.mlp_tc)) {
    // bfloat16 networks on the tensor cores: the weight gradient on the tensor cores too
    CU(tc_weight_grad(w, T, D, w->dW_stage));
    CU(cudaMemcpyAsync(dW, w->dW_stage, sizeof(float) * w->n_params, cudaMemcpyDefault, w->stream));
  } else if (dW && w->n_params > 0) {
    const size_t N = (size_t)T.horizon * w->Bp;
    const int splits = w->splits;
    const size_t chunk = ((N + splits - 1) / splits + 15) / 16 * 16;
    const int nl = T.n_layers + (T.skip ? 1 : 0);
    size_t off = 0;
    for (int l = 0; l < nl; ++l) {
      const bool sk = l == T.n_layers;
      const int ni = sk ? T.widths[0] : T.widths[l];
      const int no_ = sk ? T.widths[T.n_layers] : T.widths[l + 1];
      const float* del = D.dump + (size_t)T.dump_del[sk ? T.n_layers - 1 : l] * N;
      const float* act = D.dump + (size_t)T.dump_act[sk ? 0 : l] * N;
      CU(launch_dw(del, act, no_, ni, N, w->partial, splits, chunk, w->stream));
      CU(launch_sum_splits(w->partial, splits, (size_t)no_ * ni, w->dW_stage + off, w->stream));
      off += (size_t)no_ * ni;
      CU(launch_rowsum(del, no_, N, w->partial, splits, chunk, w->stream));
      CU(launch_sum_splits(w->partial, splits, (size_t)no_, w->dW_stage + off, w->stream));
      off += no_;
    }
    CU(cudaMemcpyAsync(dW, w->dW_stage, sizeof(float) * w->n_params, cudaMemcpyDefault, w->stream));
  }
  return DP_OK;
}

// Per-instance status words after a synchronisation of the world's stream.
static dp_status read_status(dp_world* w, std::vector<int>& st) {
  CU(cudaStreamSynchronize(w->stream));
  st.assign(w->Bp, 0);
  CU(cudaMemcpy(st.data(), w->D.status, sizeof(int) * w->Bp, cudaMemcpyDeviceToHost));
  return DP_OK;
}

dp_status dp_sync(dp_world* w) {
  if (!w) return fail(DP_EINVAL, "world is NULL");
  std::vector<int> st;
  TRY(read_status(w, st));
  for (int i = 0; i < w->B; ++i) {
    if (st[i] & DPK_ST_NAN_STATE)
      return fail(DP_ENAN, "instance " + std::to_string(i) + " produced a non-finite state or loss");
    if (st[i] & DPK_ST_NAN_GRAD)
      return fail(DP_ENAN, "instance " + std::to_string(i) + " produced a non-finite gradient");
  }
  return DP_OK;
}

dp_status dp_instance_status(dp_world* w, int32_t* status) {
  if (!w || !status) return fail(DP_EINVAL, "world or status is NULL");
  CU(cudaMemcpyAsync(status, w->D.status, sizeof(int32_t) * w->B, cudaMemcpyDefault, w->stream));
  return DP_OK;
}

dp_status dp_last_error_detail(dp_world* w, char* buf, size_t n) {
  if (!w || (!buf && n > 0)) return fail(DP_EINVAL, "world or buf is NULL");
  std::vector<int> st;
  TRY(read_status(w, st));
  std::string msg;
  int bad = 0;
  for (int bit : {DPK_ST_NAN_STATE, DPK_ST_NAN_GRAD}) {
    std::string list;
    int cnt = 0;
    for (int i = 0; i < w->B; ++i)
      if (st[i] & bit) {
        if (cnt < 8) list += (cnt ? ", " : "") + std::to_string(i);
        ++cnt;
      }
    bad += cnt;
    msg += (bit == DPK_ST_NAN_STATE ? "non-finite state or loss: " : "; non-finite gradient: ") + std::to_string(cnt) +
           " of " + std::to_string(w->B) + " instances" + (cnt ? " (" + list + (cnt > 8 ? ", ..." : "") + ")" : "");
  }
  msg += "; last error: " + g_err;
  if (n > 0) {
    const size_t k = std::min(n - 1, msg.size());
    std::memcpy(buf, msg.data(), k);
    buf[k] = '\0';
  }
  return bad ? DP_ENAN : DP_OK;
}

}  // extern "C"
