// Device-side types shared by the kernels of libdphys (not part of the public ABI).
//
// Mapping: one lane = one robot instance. A warp owns 32 instances for the whole rollout,
// so the solver's Gauss-Seidel order is executed exactly and every SIMT lane does useful
// work. Per-instance working arrays live in shared memory as [field][32 lanes]
// (bank-conflict free); per-instance parameters, constraint rows and the per-step tape live in
// global memory as [field][instance] (coalesced: a warp touches 32 consecutive floats).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define DPK_MAXB 32
#define DPK_MAXJ 32
#define DPK_MAXS 32
#define DPK_MAXP 32
#define DPK_MAXSLOT (5 * DPK_MAXJ + 2 * DPK_MAXJ + 3 * DPK_MAXS + 3 * DPK_MAXP)
#define DPK_MAXL 6
#define DPK_MAXWSG (2 * DPK_MAXJ + DPK_MAXS + DPK_MAXP)
// per-instance status bits (DevPtrs.status): non-finite state or loss in a forward launch,
// non-finite state or parameter adjoint in the last reverse pass
#define DPK_ST_NAN_STATE 1
#define DPK_ST_NAN_GRAD 2
// rows per chunk of the multi-warp reverse sweep's hand-off ring (dp_mw.cuh)
#ifndef DPK_MW_CH
#define DPK_MW_CH 20
#endif

// Flags of DevTopo.mw_slot entries (the slot index takes the low 12 bits).
#define MW_SLOT_A 0x1000
#define MW_SLOT_B 0x2000

// Warm-start group types (feature 15 of a group).
enum { WSG_GROUND = 0, WSG_PAIR = 1, WSG_JOINT = 2, WSG_HINGE = 3 };

// Row kinds (canonical slot order: joints, limits, motors, ground contacts, pair contacts).
enum { RK_JLIN = 0, RK_JANG = 1, RK_LIMIT = 2, RK_MOTOR = 3, RK_GN = 4, RK_GT = 5, RK_PN = 6, RK_PT = 7 };

// Constraint-row record in global memory, [slot][field][instance].
enum {
  RF_LIN = 0,    // 3: J_va (J_vb = -lin)
  RF_ANGA = 3,   // 3: J_wa
  RF_ANGB = 6,   // 3: J_wb
  RF_IA = 9,     // 3: I_a^-1 J_wa (world frame)
  RF_IB = 12,    // 3: I_b^-1 J_wb
  RF_MEFF = 15,  // 1: 1/(J M^-1 J^T + gamma); 0 for inactive rows (a no-op)
  RF_BIAS = 16,  // 1
  RF_BND = 17,   // 1: servo impulse bound tau_max*h (motor rows), mu (friction rows); the other
                 //    kinds have fixed bounds: joints (-inf, inf), limits and normals [0, inf)
  RF_N = 18
};

struct DevTopo {
  int B, Bp;  // instances, padded to a multiple of 32 (stride of every [field][instance] array)
  int nb, nj, ns, np, nslots;
  int iters, horizon, features, imu_body, loss_kind, loss_mode, loss_body;
  int n_layers, skip, n_params, n_motors, ctrl_round;  // ctrl_round: 1 = bfloat16 storage points
  int topo_id;  // 0: run-time topology loops; otherwise the compiled topology with this id
  int one_warp;  // 1: every launch on one warp per group (no four-warp kernels)
  int mlp_tc;   // 1: the controller is the 24-128-128-8 bfloat16 network, run on the tensor cores
  // 1: the controller is evaluated between step launches by batched tensor-core products over all
  // instances (wide bfloat16 networks); the step kernels read its output u_t and write the next
  // step's input features s_{t+1}
  int ext_ctrl, ext_k0p, ext_nop;  // padded input width (multiple of 64) and output width (8)
  int ws;       // 1: the solve starts from the learned warm start (DevPtrs.ws_tc, ws_alpha)
  float ws_alpha;  // weight of the previous step's impulses in the warm start
  int ws_net;      // 0: the network is identically zero (the damped start alpha * previous impulses)
  int n_rec;       // H: the controller's recurrent state (Eq. g): its last H inputs are h^t, its last
                   //    H outputs give h^{t+1} = tanh(.); 0 = feed-forward
  int sm_h, sm_hb; // on-chip h^t (forward) and the adjoint of h^{t+1} carried between reverse steps
  float grad_decay;  // reverse mode: state adjoint x alpha per step (section 3.2); 1 = none
  int sm_ws;    // warm-start scratch per lane: features [16], outputs [3], harvest row ids [n_wsg]
  // warm-start groups of three rows (slot -1: none): joint linear rows, hinge angular rows with
  // the motor row, contact normal/t1/t2 rows; type WSG_*
  int n_wsg;
  int8_t wsg_type[DPK_MAXWSG];
  int16_t wsg_slot[DPK_MAXWSG][3];
  int widths[DPK_MAXL + 1];
  int w_off[DPK_MAXL + 2];   // offset of layer l's W[out][in] in the flat weights (l = n_layers: skip)
  float gravity[3], dt, ground_z, beta, gamma, slop, clock_hz;
  // per-instance parameter field offsets in the [field][Bp] parameter array
  int o_mass, o_inertia, o_anchor, o_axis, o_ref, o_limit, o_motor, o_sph_off, o_sph_rad, o_sph_mu, o_sph_e,
      o_loss_point, o_loss_target, n_pfields;
  int8_t jtype[DPK_MAXJ], ja[DPK_MAXJ], jb[DPK_MAXJ], jflags[DPK_MAXJ], jmotor[DPK_MAXJ];
  int8_t motor_joint[DPK_MAXJ];
  int8_t sbody[DPK_MAXS], pk[DPK_MAXP], pl[DPK_MAXP];
  // slots (indexed by slot) and the sweep order
  uint8_t skind[DPK_MAXSLOT], sidx[DPK_MAXSLOT], ssub[DPK_MAXSLOT];
  int8_t sa[DPK_MAXSLOT], sb[DPK_MAXSLOT];
  int16_t snormal[DPK_MAXSLOT];
  int16_t order[DPK_MAXSLOT];
  // shared-memory layout per warp, in units of 32 floats (one float per lane)
  int sm_x0, sm_x, sm_xb, sm_vb, sm_iinv, sm_invm, sm_th, sm_thd, sm_ua, sm_wst, sm_wbr, sm_lam, sm_u;
  int sm_thb, sm_thdb, sm_uab, sm_wstb, sm_iinvb, sm_invmb, sm_rc, sm_sbar, sm_vw, sm_zb, sm_act[DPK_MAXL + 1], sm_rows,
      sm_total;
  int sm_ring;  // multi-warp reverse sweep: two buffers of DPK_MW_CH (j, p_bar) pairs (shares sm_vw's region)
  // multi-warp reverse pass: the warp (0..3) that owns each body's adjoint accumulators in the
  // stages outside the sweeps, and the matching body / joint (by child body) masks per warp
  int8_t mw_own[DPK_MAXB];
  uint32_t mw_bmask[4], mw_jmask[4];
  // per warp, the slots with a side it owns in slot order: slot | MW_SLOT_A (owns side a) |
  // MW_SLOT_B (owns side b)
  int16_t mw_slot[4][DPK_MAXSLOT];
  int16_t mw_nslot[4];
  // activation/delta dump offsets (rows of [feature][T*Bp]); act l = input of layer l
  int dump_act[DPK_MAXL + 1], dump_del[DPK_MAXL + 1], dump_rows;
  // tape record of one (step, warp), lanes interleaved ([field][32]): byte offsets
  //   rows   [nslots][RF_N]       float   constraint rows
  //   lam    [iters][nslots]      float   impulse after each row update
  //   viter  [iters][nb*6]        float   velocities after each sweep
  //   vminus [nb*6]               float   velocities after the external impulses
  //   br     [iters][nslots]      uint8   clamp branch (0 inside, 1 lower bound, 2 upper bound)
  //   lam0   [nslots]             float   initial impulses (warm start; only when DevTopo.ws)
  long long rec_lam, rec_viter, rec_vminus, rec_br, rec_lam0, rec_bytes;
};

// Global buffers a kernel works on.
struct DevPtrs {
  const float* prm;      // [n_pfields][Bp]
  const float* Wt;       // controller, fp32 copies of the bf16 weights, each layer [in][out]
  const float* Wn;       // same, each layer [out][in]
  const float* bias;     // controller biases, per layer [out] (then skip bias)
  const __nv_bfloat16* Wtc;  // tensor-core weight layouts (CtrlTC), when DevTopo.mlp_tc
  const __nv_bfloat16* ws_tc;  // warm-start network, tensor-core layouts (WsTC)
  const float* ws_b;           // warm-start biases (WsTC::B1, B2, B3)
  float* harvest;              // optional: harvested rows [harvest_max][19] (features, converged impulses)
  unsigned long long* harvest_count;
  long long harvest_max;
  const float* u_noise;        // optional: controller-output perturbation [T][Bp][n_motors]
  float* resid;                // optional: per-instance sum of per-step solve residuals [Bp]
  const int* hz;               // per-instance horizons [Bp]
  // wide-controller buffers (DevTopo.ext_ctrl): features of the step about to run [Bp][ext_k0p]
  // bf16, controller outputs of every step [T][Bp][ext_nop], output adjoint of the step being
  // reversed [Bp][16], input adjoint of the features [Bp][ext_k0p]
  __nv_bfloat16* s_ext;
  float* u_ext;
  float* ub_ext;
  const float* sbar_ext;
  float* lam_prev;             // impulses the last step ended with [nslots][Bp] (kept across launches)
  float* ckpt_lam;             // optional: the same at every checkpoint [n_ckpt][nslots][Bp]
  float* state;          // current state [nb*18][Bp]
  float* ckpt;           // checkpoints [n_ckpt][nb*18][Bp]
  float* seg;            // segment states for the backward [K+1][nb*18][Bp]
  float* hrec;           // the controller's recurrent state h [n_rec][Bp] between launches
  float* ckpt_h;         // h at every checkpoint [n_ckpt][n_rec][Bp] (segment recompute), or NULL
  float* rows;           // constraint rows without a tape (rows that do not fit on chip) [nslots][RF_N][Bp]
  // Per-step solver tape, tape_steps slots: the whole horizon when it fits in device memory
  // (recorded by the rollout), else one checkpoint segment (recorded by the backward pass).
  // One contiguous record per (step, warp) of rec_bytes (see DevTopo.rec_*), so a whole record
  // can be prefetched into L2 with one bulk operation.
  uint8_t* tape;
  float* dump;           // controller activations and deltas [dump_rows][T*Bp]
  float* loss;           // [Bp]
  float* dloss;          // [Bp]
  float* grad_prm;       // [n_pfields][Bp]
  float* grad_state0;    // [nb*18][Bp]
  float* traj;           // optional [T+1][B][nb][18]
  uint8_t* active;       // optional [T][B][nslots]
  int* status;           // [Bp] nonzero: non-finite value met
  int ckpt_every, n_ckpt;
  int tape_steps, tape_full;  // tape_full: the rollout records every step (no recompute)
};

// Tape record of one step for this lane's warp (pointers include the lane offset).
struct TapeStep {
  float* rows;    // field f at rows[f * 32]
  float* lam;     // (it, s) at lam[(it * nslots + s) * 32]
  float* viter;   // (it, j) at viter[(it * nb * 6 + j) * 32]
  float* vminus;  // j at vminus[j * 32]
  uint8_t* br;    // (it, s) at br[(it * nslots + s) * 32]
  float* lam0;    // s at lam0[s * 32]
  const uint8_t* rec;
};
__device__ __forceinline__ TapeStep tape_step(const DevTopo& T, const DevPtrs& D, int ts) {
  // one CTA per group of 32 instances (its warps share the group's lanes)
  const int lane = threadIdx.x & 31, warp = blockIdx.x;
  const uint8_t* rec = D.tape + ((size_t)ts * (T.Bp / 32) + warp) * (size_t)T.rec_bytes;
  TapeStep p;
  p.rec = rec;
  p.rows = (float*)rec + lane;
  p.lam = (float*)(rec + T.rec_lam) + lane;
  p.viter = (float*)(rec + T.rec_viter) + lane;
  p.vminus = (float*)(rec + T.rec_vminus) + lane;
  p.br = (uint8_t*)(rec + T.rec_br) + lane;
  p.lam0 = (float*)(rec + T.rec_lam0) + lane;
  return p;
}
// Pulls one 128-byte line (a warp's 32 contiguous lanes of one field) into L1 (fire-and-forget).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
// Pulls the 128-byte line holding p into L2 (fire-and-forget).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// Bulk prefetch of a tape record into L2 (issued by one lane; fire-and-forget).
__device__ __forceinline__ void prefetch_record_l2(const DevTopo& T, const uint8_t* rec) {
  if ((threadIdx.x & 31) != 0) return;
  for (long long off = 0; off < T.rec_bytes; off += 32768) {
    const unsigned n = (unsigned)min((long long)32768, T.rec_bytes - off);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(rec + off), "r"(n) : "memory");
  }
}

// ------------------------------------------------------------------------------- math
struct M3 { float m[9]; };

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a = a + b; return a; }
__device__ __forceinline__ float3& operator-=(float3& a, float3 b) { a = a - b; return a; }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 mv(const M3& R, float3 x) {
  return f3(R.m[0] * x.x + R.m[1] * x.y + R.m[2] * x.z, R.m[3] * x.x + R.m[4] * x.y + R.m[5] * x.z,
            R.m[6] * x.x + R.m[7] * x.y + R.m[8] * x.z);
}
__device__ __forceinline__ float3 mtv(const M3& R, float3 x) {
  return f3(R.m[0] * x.x + R.m[3] * x.y + R.m[6] * x.z, R.m[1] * x.x + R.m[4] * x.y + R.m[7] * x.z,
            R.m[2] * x.x + R.m[5] * x.y + R.m[8] * x.z);
}
__device__ __forceinline__ M3 mm(const M3& A, const M3& B) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C.m[3 * i + j] = A.m[3 * i] * B.m[j] + A.m[3 * i + 1] * B.m[3 + j] + A.m[3 * i + 2] * B.m[6 + j];
  return C;
}
__device__ __forceinline__ M3 mT(const M3& A) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.m[3 * i + j] = A.m[3 * j + i];
  return C;
}
__device__ __forceinline__ M3 eye3() {
  M3 I;
#pragma unroll
  for (int k = 0; k < 9; ++k) I.m[k] = (k % 4 == 0) ? 1.f : 0.f;
  return I;
}
// symmetric matrix stored as xx, xy, xz, yy, yz, zz
__device__ __forceinline__ float3 symv(const float* s6, float3 x) {
  return f3(s6[0] * x.x + s6[1] * x.y + s6[2] * x.z, s6[1] * x.x + s6[3] * x.y + s6[4] * x.z,
            s6[2] * x.x + s6[4] * x.y + s6[5] * x.z);
}
// R diag(d) R^T as 6 unique entries
__device__ __forceinline__ void rot_diag6(const M3& R, float3 d, float* o) {
  const float* r = R.m;
  o[0] = r[0] * r[0] * d.x + r[1] * r[1] * d.y + r[2] * r[2] * d.z;
  o[1] = r[0] * r[3] * d.x + r[1] * r[4] * d.y + r[2] * r[5] * d.z;
  o[2] = r[0] * r[6] * d.x + r[1] * r[7] * d.y + r[2] * r[8] * d.z;
  o[3] = r[3] * r[3] * d.x + r[4] * r[4] * d.y + r[5] * r[5] * d.z;
  o[4] = r[3] * r[6] * d.x + r[4] * r[7] * d.y + r[5] * r[8] * d.z;
  o[5] = r[6] * r[6] * d.x + r[7] * r[7] * d.y + r[8] * r[8] * d.z;
}
// Orthonormal basis of a unit vector (Duff et al. 2017, "Building an Orthonormal Basis,
// Revisited"), sign(0) = +1.
__device__ __forceinline__ void onb3(float3 n, float3& t1, float3& t2) {
  float s = n.z >= 0.f ? 1.f : -1.f;
  float a = -1.f / (s + n.z);
  float b = n.x * n.y * a;
  t1 = f3(1.f + s * n.x * n.x * a, s * b, -s * n.x);
  t2 = f3(b, s + n.y * n.y * a, -n.y);
}
// Reverse mode of onb3 for fixed sign: accumulate dL/dn given dL/dt1, dL/dt2.
__device__ __forceinline__ float3 onb3_vjp(float3 n, float3 g1, float3 g2) {
  float s = n.z >= 0.f ? 1.f : -1.f;
  float a = -1.f / (s + n.z);
  float a2 = a * a;  // da/dnz
  // b = nx ny a
  float db_dx = n.y * a, db_dy = n.x * a, db_dz = n.x * n.y * a2;
  float3 g = f3(0.f, 0.f, 0.f);
  // t1 = (1 + s nx^2 a, s b, -s nx)
  g.x += g1.x * (2.f * s * n.x * a) + g1.y * s * db_dx - g1.z * s;
  g.y += g1.y * s * db_dy;
  g.z += g1.x * (s * n.x * n.x * a2) + g1.y * s * db_dz;
  // t2 = (b, s + ny^2 a, -ny)
  g.x += g2.x * db_dx;
  g.y += g2.x * db_dy + g2.y * (2.f * n.y * a) - g2.z;
  g.z += g2.x * db_dz + g2.y * (n.y * n.y * a2);
  return g;
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Lane views: shared memory [field][32], global memory [field][Bp].
struct SL {
  static constexpr bool is_global = false;
  float* p;
  __device__ __forceinline__ SL at(int f) const { return SL{p + f * 32}; }
  __device__ __forceinline__ float& operator[](int f) const { return p[f * 32]; }
  // field f of lane r of this warp
  __device__ __forceinline__ float& lane_at(int f, int r) const { return p[f * 32 + r - (int)(threadIdx.x & 31)]; }
  __device__ __forceinline__ float3 v3(int f) const { return f3(p[f * 32], p[(f + 1) * 32], p[(f + 2) * 32]); }
  __device__ __forceinline__ void s3(int f, float3 v) const { p[f * 32] = v.x; p[(f + 1) * 32] = v.y; p[(f + 2) * 32] = v.z; }
  __device__ __forceinline__ void a3(int f, float3 v) const { p[f * 32] += v.x; p[(f + 1) * 32] += v.y; p[(f + 2) * 32] += v.z; }
};
// Global view with a run-time stride (f * s stays below 2^31 for every buffer indexed this way).
struct GL {
  static constexpr bool is_global = true;
  float* p;
  int s;
  __device__ __forceinline__ float& operator[](int f) const { return p[f * s]; }
  __device__ __forceinline__ float3 v3(int f) const { return f3(p[f * s], p[(f + 1) * s], p[(f + 2) * s]); }
  __device__ __forceinline__ void s3(int f, float3 v) const { p[f * s] = v.x; p[(f + 1) * s] = v.y; p[(f + 2) * s] = v.z; }
  __device__ __forceinline__ void a3(int f, float3 v) const { p[f * s] += v.x; p[(f + 1) * s] += v.y; p[(f + 2) * s] += v.z; }
  __device__ __forceinline__ GL at(int f) const { return GL{p + f * s, s}; }
  // fire-and-forget accumulation (a reduction whose result is not read back): no load latency;
  // each lane owns its addresses, and one thread's reductions to one address apply in order
  __device__ __forceinline__ void red(int f, float v) const { atomicAdd(p + f * s, v); }
  __device__ __forceinline__ void red3(int f, float3 v) const {
    atomicAdd(p + f * s, v.x);
    atomicAdd(p + (f + 1) * s, v.y);
    atomicAdd(p + (f + 2) * s, v.z);
  }
};
// Global view with the lane-interleaved layout of shared memory (stride 32): tape records.
struct GS {
  static constexpr bool is_global = true;
  float* p;
  __device__ __forceinline__ GS at(int f) const { return GS{p + f * 32}; }
  __device__ __forceinline__ float& operator[](int f) const { return p[f * 32]; }
  __device__ __forceinline__ float3 v3(int f) const { return f3(p[f * 32], p[(f + 1) * 32], p[(f + 2) * 32]); }
  __device__ __forceinline__ void s3(int f, float3 v) const { p[f * 32] = v.x; p[(f + 1) * 32] = v.y; p[(f + 2) * 32] = v.z; }
};
// Read-only tape view (non-coherent loads: the record was written by an earlier kernel).
struct GSR {
  static constexpr bool is_global = true;
  const float* p;
  __device__ __forceinline__ GSR at(int f) const { return GSR{p + f * 32}; }
  __device__ __forceinline__ float operator[](int f) const { return __ldg(p + f * 32); }
  __device__ __forceinline__ float3 v3(int f) const { return f3(__ldg(p + f * 32), __ldg(p + (f + 1) * 32), __ldg(p + (f + 2) * 32)); }
};
// Wide-stride global view (controller activation/delta columns of the [row][T*Bp] dump).
struct GW {
  float* p;
  size_t s;
  __device__ __forceinline__ float& operator[](int f) const { return p[(size_t)f * s]; }
  __device__ __forceinline__ float& lane_at(int f, int r) const { return p[(size_t)f * s + r - (int)(threadIdx.x & 31)]; }
};
struct GC {
  const float* p;
  int s;
  __device__ __forceinline__ float operator[](int f) const { return __ldg(p + f * s); }
  __device__ __forceinline__ float3 v3(int f) const { return f3((*this)[f], (*this)[f + 1], (*this)[f + 2]); }
};

template <class XV>
__device__ __forceinline__ M3 loadRv(const XV& X, int base) {
  M3 R;
#pragma unroll
  for (int k = 0; k < 9; ++k) R.m[k] = X[base + 3 + k];
  return R;
}
__device__ __forceinline__ M3 loadR(const SL& X, int base) {
  M3 R;
#pragma unroll
  for (int k = 0; k < 9; ++k) R.m[k] = X[base + 3 + k];
  return R;
}
