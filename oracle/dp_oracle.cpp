// FP64 CPU oracle for the differentiable rigid-body step of
// "A Differentiable Physics Engine for Deep Learning in Robotics" (arXiv 1611.01652).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path links, imports or calls this file;
// only the test-suite, the smoke check and the CPU-baseline leg of the benchmark do.
// It shares no code, header, table or constant with the CUDA library.
//
// What it computes (paper section 2.1 "A 3D Rigid Body Engine"):
//   * bodies with 6 DoF whose orientation is a rotation matrix, renormalised every step
//     with the update of Eq. 1 (read as the polar / Newton-Schulz step A' = (3A - A A^T A)/2,
//     because the printed elementwise form does not keep a rotation fixed);
//   * constraints between bodies (ball and hinge joints, joint limits, servo motors,
//     sphere-ground and sphere-sphere contacts with Coulomb friction and restitution),
//     softened as in the sequential-impulse formulation the paper cites;
//   * a fixed number of projected Gauss-Seidel sweeps for the constraint impulses;
//   * semi-implicit Euler: the new velocities are integrated to give the new positions;
//   * branchless sphere contact detection (every slot is evaluated, inactive slots are masked);
//   * servo motors with gain, maximal torque and maximal velocity.
// The controller is the dense policy of Eq. g (section 2.2), optionally with its recurrent
// state h^t (h^0 = 0): the network reads [features, h^t] and its last outputs, through tanh,
// give h^{t+1}; the rollout loss is Eq. L. Gradients are reverse mode through the whole rollout
// (section 2.1.1, back-propagation through time), obtained here with a plain operator-
// overloading tape that records every arithmetic operation of one step.
//
// Every formula the paper does not print is a stated reading; the readings are listed in
// the repository's design notes and repeated next to the code that takes them.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc {

// ----------------------------------------------------------------------------------------
// Reverse-mode tape: each node has up to two parents and the local partials.
struct Tape {
  std::vector<int32_t> pa, pb;
  std::vector<double> da, db;
  std::vector<double> adj;
  void clear() { pa.clear(); pb.clear(); da.clear(); db.clear(); adj.clear(); }
  int32_t push(int32_t a, double ga, int32_t b, double gb) {
    pa.push_back(a); da.push_back(ga); pb.push_back(b); db.push_back(gb);
    return (int32_t)pa.size() - 1;
  }
  void backward() {
    for (int64_t i = (int64_t)pa.size() - 1; i >= 0; --i) {
      double g = adj[i];
      if (g == 0.0) continue;
      if (pa[i] >= 0) adj[pa[i]] += da[i] * g;
      if (pb[i] >= 0) adj[pb[i]] += db[i] * g;
    }
  }
};
static thread_local Tape* g_tape = nullptr;

struct AD {
  double v;
  int32_t id;
  AD() : v(0.0), id(-1) {}
  AD(double x) : v(x), id(-1) {}
  AD(double x, int32_t i) : v(x), id(i) {}
};
static inline AD mk(double v, int32_t a, double ga, int32_t b, double gb) {
  if (a < 0 && b < 0) return AD(v);
  return AD(v, g_tape->push(a, ga, b, gb));
}
static inline AD leaf(double v) { return AD(v, g_tape->push(-1, 0.0, -1, 0.0)); }
inline AD operator+(AD a, AD b) { return mk(a.v + b.v, a.id, 1.0, b.id, 1.0); }
inline AD operator-(AD a, AD b) { return mk(a.v - b.v, a.id, 1.0, b.id, -1.0); }
inline AD operator*(AD a, AD b) { return mk(a.v * b.v, a.id, b.v, b.id, a.v); }
inline AD operator/(AD a, AD b) {
  double r = a.v / b.v;
  return mk(r, a.id, 1.0 / b.v, b.id, -r / b.v);
}
inline AD operator-(AD a) { return mk(-a.v, a.id, -1.0, -1, 0.0); }
inline AD& operator+=(AD& a, AD b) { a = a + b; return a; }
inline AD& operator-=(AD& a, AD b) { a = a - b; return a; }
inline AD& operator*=(AD& a, AD b) { a = a * b; return a; }
inline AD sqrt(AD a) {
  double r = std::sqrt(a.v);
  return mk(r, a.id, 0.5 / r, -1, 0.0);
}
inline AD sin(AD a) { return mk(std::sin(a.v), a.id, std::cos(a.v), -1, 0.0); }
inline AD cos(AD a) { return mk(std::cos(a.v), a.id, -std::sin(a.v), -1, 0.0); }
inline AD atan2(AD y, AD x) {
  double d = x.v * x.v + y.v * y.v;
  return mk(std::atan2(y.v, x.v), y.id, x.v / d, x.id, -y.v / d);
}
inline AD tanh(AD a) {
  double r = std::tanh(a.v);
  return mk(r, a.id, 1.0 - r * r, -1, 0.0);
}

// Counting scalar: every arithmetic operation and elementary function adds one to g_flops
// (the instrumented counter that gives the algorithmic work of one step).
static thread_local double g_flops = 0.0;
struct CNT {
  double v;
  CNT() : v(0.0) {}
  CNT(double x) : v(x) {}
};
inline CNT operator+(CNT a, CNT b) { g_flops += 1; return CNT(a.v + b.v); }
inline CNT operator-(CNT a, CNT b) { g_flops += 1; return CNT(a.v - b.v); }
inline CNT operator*(CNT a, CNT b) { g_flops += 1; return CNT(a.v * b.v); }
inline CNT operator/(CNT a, CNT b) { g_flops += 1; return CNT(a.v / b.v); }
inline CNT operator-(CNT a) { return CNT(-a.v); }
inline CNT& operator+=(CNT& a, CNT b) { a = a + b; return a; }
inline CNT& operator-=(CNT& a, CNT b) { a = a - b; return a; }
inline CNT& operator*=(CNT& a, CNT b) { a = a * b; return a; }
inline CNT sqrt(CNT a) { g_flops += 1; return CNT(std::sqrt(a.v)); }
inline CNT sin(CNT a) { g_flops += 1; return CNT(std::sin(a.v)); }
inline CNT cos(CNT a) { g_flops += 1; return CNT(std::cos(a.v)); }
inline CNT atan2(CNT y, CNT x) { g_flops += 1; return CNT(std::atan2(y.v, x.v)); }
inline CNT tanh(CNT a) { g_flops += 1; return CNT(std::tanh(a.v)); }

inline double val(double x) { return x; }
inline double val(const AD& x) { return x.v; }
inline double val(const CNT& x) { return x.v; }
using std::sqrt;
using std::sin;
using std::cos;
using std::atan2;
using std::tanh;

// Round to bfloat16 (8 significant bits), round-to-nearest-even. Straight-through
// derivative for the AD type (the rounding is treated as the identity in reverse mode).
double bf16(double x) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e;
  double m = std::frexp(x, &e);       // |m| in [0.5, 1)
  double s = std::ldexp(m, 8);        // |s| in [128, 256)
  double r = std::nearbyint(s);       // default rounding mode: ties to even
  return std::ldexp(r, e - 8);
}
static thread_local bool g_exact_mlp = false;
// Smallest relative distance, over the roundings of one step, of a pre-rounding value to a
// bfloat16 rounding midpoint (how close a quantisation decision came to flipping).
static thread_local double g_bf16_margin = INFINITY;
inline double bf16_tie_distance(double x) {
  if (x == 0.0 || !std::isfinite(x)) return INFINITY;
  int e;
  double m = std::frexp(x, &e);
  double s = std::ldexp(std::fabs(m), 8);  // [128, 256)
  double frac = s - std::floor(s);
  return std::fabs(frac - 0.5) / s;
}
inline double round_bf16(double x) {
  if (g_exact_mlp) return x;
  g_bf16_margin = std::min(g_bf16_margin, bf16_tie_distance(x));
  return bf16(x);
}
inline CNT round_bf16(CNT x) { return CNT(g_exact_mlp ? x.v : bf16(x.v)); }
inline CNT round_bf16_w(CNT x) { return round_bf16(x); }
inline AD round_bf16(AD x) { return g_exact_mlp ? x : mk(bf16(x.v), x.id, 1.0, -1, 0.0); }
// Weights are exact float32 inputs on every side, so their rounding is not a tie risk.
inline double round_bf16_w(double x) { return g_exact_mlp ? x : bf16(x); }
inline AD round_bf16_w(AD x) { return round_bf16(x); }

// Branch helpers: the branch is chosen on the value; ties go to the stated side.
template <class S> inline S clamp_sel(S x, S lo, S hi, int* branch) {
  if (val(x) < val(lo)) { if (branch) *branch = 1; return lo; }
  if (val(x) > val(hi)) { if (branch) *branch = 2; return hi; }
  if (branch) *branch = 0;
  return x;
}
template <class S> inline S min0(S x) { return val(x) < 0.0 ? x : S(0.0); }   // min(x, 0), tie -> 0
template <class S> inline S relu(S x) { return val(x) > 0.0 ? x : S(0.0); }

// ----------------------------------------------------------------------------------------
// Small vector algebra (row-major 3x3).
template <class S> using V3 = std::array<S, 3>;
template <class S> using M3 = std::array<S, 9>;

template <class S> inline V3<S> vadd(const V3<S>& a, const V3<S>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
template <class S> inline V3<S> vsub(const V3<S>& a, const V3<S>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
template <class S> inline V3<S> vscale(const V3<S>& a, S s) { return {a[0] * s, a[1] * s, a[2] * s}; }
template <class S> inline V3<S> vneg(const V3<S>& a) { return {-a[0], -a[1], -a[2]}; }
template <class S> inline S dot(const V3<S>& a, const V3<S>& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class S> inline V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
template <class S> inline V3<S> matvec(const M3<S>& m, const V3<S>& x) {
  return {m[0] * x[0] + m[1] * x[1] + m[2] * x[2], m[3] * x[0] + m[4] * x[1] + m[5] * x[2],
          m[6] * x[0] + m[7] * x[1] + m[8] * x[2]};
}
template <class S> inline V3<S> matTvec(const M3<S>& m, const V3<S>& x) {
  return {m[0] * x[0] + m[3] * x[1] + m[6] * x[2], m[1] * x[0] + m[4] * x[1] + m[7] * x[2],
          m[2] * x[0] + m[5] * x[1] + m[8] * x[2]};
}
template <class S> inline M3<S> matmul(const M3<S>& a, const M3<S>& b) {
  M3<S> c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
  return c;
}
template <class S> inline M3<S> transpose(const M3<S>& a) {
  return {a[0], a[3], a[6], a[1], a[4], a[7], a[2], a[5], a[8]};
}
template <class S> inline M3<S> identity() { return {S(1.0), S(0.0), S(0.0), S(0.0), S(1.0), S(0.0), S(0.0), S(0.0), S(1.0)}; }
// R diag(d) R^T
template <class S> inline M3<S> rotate_diag(const M3<S>& R, const V3<S>& d) {
  M3<S> RD;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) RD[3 * i + j] = R[3 * i + j] * d[j];
  return matmul(RD, transpose(R));
}

// Orthonormal basis of a unit vector n: Duff et al. 2017, "Building an Orthonormal Basis,
// Revisited" (JCGT 6(1)), with sign(0) = +1.
template <class S> inline void onb(const V3<S>& n, V3<S>& t1, V3<S>& t2) {
  double sg = val(n[2]) >= 0.0 ? 1.0 : -1.0;
  S a = S(-1.0) / (S(sg) + n[2]);
  S b = n[0] * n[1] * a;
  t1 = {S(1.0) + S(sg) * n[0] * n[0] * a, S(sg) * b, S(-sg) * n[0]};
  t2 = {b, S(sg) + n[1] * n[1] * a, -n[1]};
}

}  // namespace orc

// ----------------------------------------------------------------------------------------
// C interface (consumed through ctypes by the tests).
extern "C" {

// Row kinds, in the canonical slot order of one instance.
enum { ORC_JLIN = 0, ORC_JANG = 1, ORC_LIMIT = 2, ORC_MOTOR = 3, ORC_GN = 4, ORC_GT = 5, ORC_PN = 6, ORC_PT = 7 };
enum { ORC_BALL = 0, ORC_HINGE = 1 };
enum { ORC_FLAG_LIMIT = 1, ORC_FLAG_MOTOR = 2 };
enum { ORC_F_ANGLES = 1, ORC_F_RATES = 2, ORC_F_CLOCK = 4, ORC_F_IMU = 8, ORC_F_TARGET = 16 };
enum { ORC_L_SQDIST = 0, ORC_L_DIST = 1, ORC_L_LINEAR = 2, ORC_L_DISP = 3 };
enum { ORC_M_FINAL = 0, ORC_M_MEAN = 1 };

typedef struct {
  int32_t nb, nj, ns, np;
  const int32_t* joint_type;   // [nj]
  const int32_t* joint_body;   // [nj][2]  parent a (-1 = world), child b
  const int32_t* joint_flags;  // [nj]     bit0 limit, bit1 motor (hinges only)
  const int32_t* sphere_body;  // [ns]
  const int32_t* pair_sphere;  // [np][2]
  int32_t n_layers;            // dense layers of the controller (0 = no controller)
  const int32_t* widths;       // [n_layers + 1]
  int32_t skip;                // output layer also reads the input layer
  int32_t features;            // ORC_F_* bit mask
  int32_t imu_body;
  double clock_hz;
  double gravity[3];
  double dt, ground_z, beta, gamma, slop;
  int32_t iters;
  int32_t loss_kind, loss_mode, loss_body;
  int32_t exact_mlp;           // 1: skip the bfloat16 rounding (finite-difference checks only)
  int32_t warmstart;           // 1: the solve starts from the learned warm start (ws_W, ws_alpha)
  const double* ws_W;          // warm-start network parameters [ORC_WS_PARAMS]
  double ws_alpha;             // weight of the previous step's impulses in the warm start
  double grad_decay;           // section 3.2: adjoint passed from step t+1 back to step t times alpha
  int32_t n_recurrent;         // H: recurrent state of the controller (Eq. g), the last H inputs and
                               //    outputs of the network; 0 = feed-forward
} orc_topo;

// Learned warm start: a 16-64-64-3 network per contact (W1, b1, W2, b2, W3, b3; W[out][in]).
enum { ORC_WS_IN = 16, ORC_WS_H = 64, ORC_WS_OUT = 3,
       ORC_WS_PARAMS = ORC_WS_IN * ORC_WS_H + ORC_WS_H + ORC_WS_H * ORC_WS_H + ORC_WS_H + ORC_WS_H * ORC_WS_OUT + ORC_WS_OUT };

typedef struct {
  const double* mass;         // [nb]
  const double* inertia;      // [nb][3]  principal moments in the body frame
  const double* anchor;       // [nj][2][3]
  const double* axis;         // [nj][2][3]
  const double* ref;          // [nj][2][3]
  const double* limit;        // [nj][2]
  const double* motor;        // [nj][3]  gain, max torque, max velocity
  const double* sph_off;      // [ns][3]
  const double* sph_rad;      // [ns]
  const double* sph_mu;       // [ns]
  const double* sph_e;        // [ns]
  const double* loss_point;   // [3]
  const double* loss_target;  // [3]
  const double* state0;       // [nb][18]  p, R (row-major), v, w
} orc_inst;

typedef struct {  // gradient outputs, same shapes as orc_inst (+ controller); NULL = not wanted
  double *mass, *inertia, *anchor, *axis, *ref, *limit, *motor, *sph_off, *sph_rad, *sph_mu, *sph_e,
      *loss_point, *loss_target, *state0, *W;
} orc_grad;

}  // extern "C"

namespace orc {

struct Slot {
  int kind, idx, sub, a, b, normal;
};

static std::vector<Slot> make_slots(const orc_topo& T) {
  std::vector<Slot> s;
  for (int j = 0; j < T.nj; ++j) {
    int a = T.joint_body[2 * j], b = T.joint_body[2 * j + 1];
    for (int k = 0; k < 3; ++k) s.push_back({ORC_JLIN, j, k, a, b, -1});
    if (T.joint_type[j] == ORC_HINGE)
      for (int k = 0; k < 2; ++k) s.push_back({ORC_JANG, j, k, a, b, -1});
  }
  for (int j = 0; j < T.nj; ++j)
    if (T.joint_type[j] == ORC_HINGE && (T.joint_flags[j] & ORC_FLAG_LIMIT))
      s.push_back({ORC_LIMIT, j, 0, T.joint_body[2 * j], T.joint_body[2 * j + 1], -1});
  for (int j = 0; j < T.nj; ++j)
    if (T.joint_type[j] == ORC_HINGE && (T.joint_flags[j] & ORC_FLAG_MOTOR))
      s.push_back({ORC_MOTOR, j, 0, T.joint_body[2 * j], T.joint_body[2 * j + 1], -1});
  for (int q = 0; q < T.ns; ++q) {
    int n = (int)s.size();
    s.push_back({ORC_GN, q, 0, T.sphere_body[q], -1, -1});
    s.push_back({ORC_GT, q, 0, T.sphere_body[q], -1, n});
    s.push_back({ORC_GT, q, 1, T.sphere_body[q], -1, n});
  }
  for (int q = 0; q < T.np; ++q) {
    int n = (int)s.size();
    int a = T.sphere_body[T.pair_sphere[2 * q]], b = T.sphere_body[T.pair_sphere[2 * q + 1]];
    s.push_back({ORC_PN, q, 0, a, b, -1});
    s.push_back({ORC_PT, q, 0, a, b, n});
    s.push_back({ORC_PT, q, 1, a, b, n});
  }
  return s;
}

// Greedy colouring in slot order (smallest colour not used by an earlier slot sharing a
// non-world body); sweep order = (colour ascending, slot ascending).
static void make_schedule(const std::vector<Slot>& s, std::vector<int>& colour, std::vector<int>& order) {
  int n = (int)s.size();
  colour.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    std::vector<char> used(n + 1, 0);
    for (int k = 0; k < i; ++k) {
      bool share = (s[i].a >= 0 && (s[i].a == s[k].a || s[i].a == s[k].b)) ||
                   (s[i].b >= 0 && (s[i].b == s[k].a || s[i].b == s[k].b));
      if (share) used[colour[k]] = 1;
    }
    int c = 0;
    while (used[c]) ++c;
    colour[i] = c;
  }
  order.resize(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return colour[x] < colour[y]; });
}

// Warm-start groups of three rows, in slot order of their first row: the linear rows of each
// joint (x, y, z), the angular rows of each hinge with its motor row (slot -1 without a motor),
// and the normal, t1, t2 rows of each contact.
enum { WS_GROUND = 0, WS_PAIR = 1, WS_JOINT = 2, WS_HINGE = 3 };
struct WsGroup {
  int type, slot[3];
};
static std::vector<WsGroup> ws_groups(const orc_topo& T, const std::vector<Slot>& s) {
  std::vector<WsGroup> g;
  const int n = (int)s.size();
  for (int i = 0; i < n; ++i) {
    if (s[i].kind == ORC_JLIN && s[i].sub == 0) {
      g.push_back({WS_JOINT, {i, i + 1, i + 2}});
    } else if (s[i].kind == ORC_JANG && s[i].sub == 0) {
      int motor = -1;
      for (int k = 0; k < n; ++k)
        if (s[k].kind == ORC_MOTOR && s[k].idx == s[i].idx) motor = k;
      g.push_back({WS_HINGE, {i, i + 1, motor}});
    } else if (s[i].kind == ORC_GN) {
      g.push_back({WS_GROUND, {i, i + 1, i + 2}});
    } else if (s[i].kind == ORC_PN) {
      g.push_back({WS_PAIR, {i, i + 1, i + 2}});
    }
  }
  return g;
}

template <class S> struct Inst {
  std::vector<S> mass, inertia, anchor, axis, ref, limit, motor, sph_off, sph_rad, sph_mu, sph_e, loss_point, loss_target;
};

template <class S> static std::vector<S> lift(const double* p, size_t n) {
  std::vector<S> out(n);
  for (size_t i = 0; i < n; ++i) out[i] = S(p ? p[i] : 0.0);
  return out;
}
static std::vector<AD> lift_leaf(const double* p, size_t n) {
  std::vector<AD> out(n);
  for (size_t i = 0; i < n; ++i) out[i] = leaf(p ? p[i] : 0.0);
  return out;
}

template <class S> static V3<S> get3(const std::vector<S>& v, size_t off) { return {v[off], v[off + 1], v[off + 2]}; }

int param_count(int n_layers, const int32_t* widths, int skip) {
  if (n_layers <= 0) return 0;
  int n = 0;
  for (int l = 0; l < n_layers; ++l) n += widths[l] * widths[l + 1] + widths[l + 1];
  if (skip) n += widths[0] * widths[n_layers] + widths[n_layers];
  return n;
}

int feature_count(const orc_topo& T, int n_motors) {
  int n = 0;
  if (T.features & ORC_F_ANGLES) n += n_motors;
  if (T.features & ORC_F_RATES) n += n_motors;
  if (T.features & ORC_F_CLOCK) n += 2;
  if (T.features & ORC_F_IMU) n += 6;
  if (T.features & ORC_F_TARGET) n += 3;
  return n;
}

// Per-step record used by tests: slot activity and the distance of each activation decision
// from its threshold (contacts: |gap|, limits: distance of the angle to the nearer bound).
struct StepLog {
  int8_t* active;
  double* gap;
  double* lambda;       // final impulses per slot
  double* bf16_margin;  // see g_bf16_margin
  double* resid;        // RMS complementarity residual of the solve over the active rows
  double* feats;        // [groups][ORC_WS_IN] warm-start features of every group
  double* lam0;         // [n_slots] initial impulses of the solve
};

// The warm-start network on one feature vector: inputs, weights and hidden activations stored
// in bfloat16, fp32 biases, ReLU hidden layers, linear output.
template <class S, class SW>
static void ws_forward(const SW* W, const S* x, S* y) {
  const int I = ORC_WS_IN, H = ORC_WS_H, O = ORC_WS_OUT;
  const SW* W1 = W;
  const SW* b1 = W1 + I * H;
  const SW* W2 = b1 + H;
  const SW* b2 = W2 + H * H;
  const SW* W3 = b2 + H;
  const SW* b3 = W3 + H * O;
  S xi[ORC_WS_IN], h1[ORC_WS_H], h2[ORC_WS_H];
  for (int i = 0; i < I; ++i) xi[i] = round_bf16(x[i]);
  for (int o = 0; o < H; ++o) {
    S acc = b1[o];
    for (int i = 0; i < I; ++i) acc += round_bf16_w(W1[o * I + i]) * xi[i];
    h1[o] = round_bf16(relu(acc));
  }
  for (int o = 0; o < H; ++o) {
    S acc = b2[o];
    for (int i = 0; i < H; ++i) acc += round_bf16_w(W2[o * H + i]) * h1[i];
    h2[o] = round_bf16(relu(acc));
  }
  for (int o = 0; o < O; ++o) {
    S acc = b3[o];
    for (int i = 0; i < H; ++i) acc += round_bf16_w(W3[o * H + i]) * h2[i];
    y[o] = acc;
  }
}

// The loss point q = p_b + R_b c of the body named by loss_body.
template <class S> static V3<S> loss_point_of(const orc_topo& T, const Inst<S>& P, const std::vector<S>& x) {
  int b = T.loss_body;
  V3<S> p = get3(x, 18 * b);
  M3<S> R;
  for (int k = 0; k < 9; ++k) R[k] = x[18 * b + 3 + k];
  return vadd(p, matvec(R, get3(P.loss_point, 0)));
}
// l(x) of Eq. L for one state (the displacement kind contributes a.q here and -a.q_0 once).
template <class S> static S loss_of(const orc_topo& T, const Inst<S>& P, const std::vector<S>& x) {
  V3<S> q = loss_point_of(T, P, x);
  V3<S> tg = get3(P.loss_target, 0);
  switch (T.loss_kind) {
    case ORC_L_SQDIST: { V3<S> d = vsub(q, tg); return dot(d, d); }
    case ORC_L_DIST: { V3<S> d = vsub(q, tg); return sqrt(dot(d, d)); }
    default: return dot(tg, q);
  }
}
template <class S> static S loss_initial(const orc_topo& T, const Inst<S>& P, const std::vector<S>& x0) {
  if (T.loss_kind != ORC_L_DISP) return S(0.0);
  return -dot(get3(P.loss_target, 0), loss_point_of(T, P, x0));
}

// One time step x_t -> x_{t+1} (section 2.1, steps in the order the paper describes them:
// controller, forces, constraints (LCP) solved by projected Gauss-Seidel, then semi-implicit
// Euler). Returns the loss contribution of x_{t+1} (weight w_next) in *loss.
template <class S>
static void step(const orc_topo& T, const std::vector<Slot>& slots, const std::vector<int>& order, const Inst<S>& P,
                 const std::vector<S>& W, int t, const std::vector<S>& x, std::vector<S>& xn, double w_next, S* loss,
                 StepLog* log, const double* lam_prev = nullptr, double* lam_out = nullptr,
                 const std::vector<S>* h_in = nullptr, std::vector<S>* h_out = nullptr) {
  const double h = T.dt;
  const int nb = T.nb, nj = T.nj;
  g_exact_mlp = T.exact_mlp != 0;
  g_bf16_margin = INFINITY;
  std::vector<V3<S>> p(nb), v(nb), w(nb);
  std::vector<M3<S>> R(nb);
  for (int b = 0; b < nb; ++b) {
    p[b] = get3(x, 18 * b);
    for (int k = 0; k < 9; ++k) R[b][k] = x[18 * b + 3 + k];
    v[b] = get3(x, 18 * b + 12);
    w[b] = get3(x, 18 * b + 15);
  }
  auto Rof = [&](int b) { return b < 0 ? identity<S>() : R[b]; };
  auto pof = [&](int b) { return b < 0 ? V3<S>{S(0.0), S(0.0), S(0.0)} : p[b]; };
  auto wof = [&](int b) { return b < 0 ? V3<S>{S(0.0), S(0.0), S(0.0)} : w[b]; };

  // Hinge geometry at x_t: axis u_a = R_a axis_a, angle about it (atan2 of the two reference
  // vectors) and its rate u_a . (w_b - w_a).
  std::vector<S> theta(nj, S(0.0)), thetadot(nj, S(0.0));
  std::vector<V3<S>> ua(nj);
  for (int j = 0; j < nj; ++j) {
    int a = T.joint_body[2 * j], b = T.joint_body[2 * j + 1];
    ua[j] = matvec(Rof(a), get3(P.axis, 6 * j));
    if (T.joint_type[j] != ORC_HINGE) continue;
    V3<S> wa = matvec(Rof(a), get3(P.ref, 6 * j));
    V3<S> wb = matvec(Rof(b), get3(P.ref, 6 * j + 3));
    theta[j] = atan2(dot(cross(wa, wb), ua[j]), dot(wa, wb));
    thetadot[j] = dot(ua[j], vsub(wof(b), wof(a)));
  }
  std::vector<int> motors;
  for (int j = 0; j < nj; ++j)
    if (T.joint_type[j] == ORC_HINGE && (T.joint_flags[j] & ORC_FLAG_MOTOR)) motors.push_back(j);

  // Controller (Eq. g): [features, h^t] -> dense ReLU layers -> linear output; the first outputs
  // are the motor signals u^t, the last H give the next recurrent state h^{t+1} = tanh(.).
  // bfloat16 storage points: the input vector (h^t included), every weight, every hidden
  // activation; h^{t+1} itself is kept in full precision.
  std::vector<S> u(motors.size(), S(0.0));
  const int H = T.n_recurrent;
  if (h_out) h_out->assign(H, S(0.0));
  if (T.n_layers > 0) {
    std::vector<S> s;
    if (T.features & ORC_F_ANGLES) for (int j : motors) s.push_back(theta[j]);
    if (T.features & ORC_F_RATES) for (int j : motors) s.push_back(thetadot[j]);
    if (T.features & ORC_F_CLOCK) {
      double ph = 2.0 * M_PI * T.clock_hz * (t * h);
      s.push_back(S(std::sin(ph)));
      s.push_back(S(std::cos(ph)));
    }
    if (T.features & ORC_F_IMU) {
      int b = T.imu_body;
      V3<S> g = matTvec(R[b], V3<S>{S(0.0), S(0.0), S(-1.0)});
      V3<S> wl = matTvec(R[b], w[b]);
      for (int k = 0; k < 3; ++k) s.push_back(g[k]);
      for (int k = 0; k < 3; ++k) s.push_back(wl[k]);
    }
    if (T.features & ORC_F_TARGET) {
      V3<S> d = vsub(loss_point_of(T, P, x), get3(P.loss_target, 0));
      for (int k = 0; k < 3; ++k) s.push_back(d[k]);
    }
    s.resize(T.widths[0] - H, S(0.0));
    for (int k = 0; k < H; ++k) s.push_back(h_in ? (*h_in)[k] : S(0.0));
    for (auto& e : s) e = round_bf16(e);
    std::vector<S> a = s;
    size_t off = 0;
    for (int l = 0; l < T.n_layers; ++l) {
      int ni = T.widths[l], no = T.widths[l + 1];
      std::vector<S> z(no);
      for (int o = 0; o < no; ++o) {
        S acc = W[off + (size_t)ni * no + o];  // bias (kept in fp32)
        for (int i = 0; i < ni; ++i) acc += round_bf16_w(W[off + (size_t)o * ni + i]) * a[i];
        z[o] = acc;
      }
      off += (size_t)ni * no + no;
      if (l + 1 < T.n_layers) {
        for (int o = 0; o < no; ++o) z[o] = round_bf16(relu(z[o]));
      } else if (T.skip) {
        for (int o = 0; o < no; ++o) {
          S acc = W[off + (size_t)T.widths[0] * no + o];  // skip-layer bias
          for (int i = 0; i < T.widths[0]; ++i) acc += round_bf16_w(W[off + (size_t)o * T.widths[0] + i]) * s[i];
          z[o] += acc;
        }
      }
      a = z;
    }
    for (size_t m = 0; m < motors.size() && m < a.size(); ++m) u[m] = a[m];
    if (h_out)
      for (int k = 0; k < H; ++k) (*h_out)[k] = tanh(a[a.size() - H + k]);
  }

  // Servo: target joint rate w* = clamp(k (u - theta), -vmax, vmax).
  std::vector<S> wstar(nj, S(0.0));
  for (size_t m = 0; m < motors.size(); ++m) {
    int j = motors[m];
    S k = P.motor[3 * j], vmax = P.motor[3 * j + 2];
    wstar[j] = clamp_sel(k * (u[m] - theta[j]), -vmax, vmax, (int*)nullptr);
  }

  // External impulses: gravity, and the explicit gyroscopic term w += h I^-1 (-(w x I w)).
  std::vector<S> invm(nb);
  std::vector<M3<S>> Iinv(nb);
  for (int b = 0; b < nb; ++b) {
    invm[b] = S(1.0) / P.mass[b];
    V3<S> I = get3(P.inertia, 3 * b);
    V3<S> Ii = {S(1.0) / I[0], S(1.0) / I[1], S(1.0) / I[2]};
    M3<S> Iw = rotate_diag(R[b], I);
    Iinv[b] = rotate_diag(R[b], Ii);
    v[b] = vadd(v[b], vscale(V3<S>{S(T.gravity[0]), S(T.gravity[1]), S(T.gravity[2])}, S(h)));
    V3<S> gyro = vneg(cross(w[b], matvec(Iw, w[b])));
    w[b] = vadd(w[b], vscale(matvec(Iinv[b], gyro), S(h)));
  }
  auto vof = [&](int b) { return b < 0 ? V3<S>{S(0.0), S(0.0), S(0.0)} : v[b]; };
  auto wvof = [&](int b) { return b < 0 ? V3<S>{S(0.0), S(0.0), S(0.0)} : w[b]; };

  // Constraint rows (Jacobian J = [lin, angA, -lin, angB], effective mass, bias, bounds).
  const int ns_ = (int)slots.size();
  struct Row {
    bool active;
    int a, b, normal;
    V3<S> lin, angA, angB;
    S meff, bias, lo, hi, mu;
    bool friction;
  };
  std::vector<Row> rows(ns_);
  const double bh = T.beta / h;
  const V3<S> ez = {S(0.0), S(0.0), S(1.0)};
  for (int si = 0; si < ns_; ++si) {
    const Slot& sl = slots[si];
    Row r;
    r.a = sl.a; r.b = sl.b; r.normal = sl.normal;
    r.active = true; r.friction = false;
    r.lin = {S(0.0), S(0.0), S(0.0)}; r.angA = r.lin; r.angB = r.lin;
    r.bias = S(0.0); r.lo = S(-INFINITY); r.hi = S(INFINITY); r.mu = S(0.0);
    double gap = INFINITY;
    switch (sl.kind) {
      case ORC_JLIN: {
        int j = sl.idx;
        V3<S> ra = matvec(Rof(sl.a), get3(P.anchor, 6 * j));
        V3<S> rb = matvec(Rof(sl.b), get3(P.anchor, 6 * j + 3));
        V3<S> C = vsub(vadd(pof(sl.a), ra), vadd(pof(sl.b), rb));
        V3<S> e = {S(0.0), S(0.0), S(0.0)};
        e[sl.sub] = S(1.0);
        r.lin = e;
        r.angA = cross(ra, e);
        r.angB = vneg(cross(rb, e));
        r.bias = S(bh) * C[sl.sub];
        break;
      }
      case ORC_JANG: {
        // Tangents fixed in the parent frame: basis of the static axis, rotated by R_a.
        int j = sl.idx;
        V3<S> t1, t2;
        onb(get3(P.axis, 6 * j), t1, t2);
        V3<S> tk = matvec(Rof(sl.a), sl.sub == 0 ? t1 : t2);
        V3<S> ubv = matvec(Rof(sl.b), get3(P.axis, 6 * j + 3));
        r.angA = tk;
        r.angB = vneg(tk);
        r.bias = S(bh) * dot(tk, cross(ubv, ua[j]));  // C with dC/dt = J v
        break;
      }
      case ORC_LIMIT: {
        int j = sl.idx;
        S lo = P.limit[2 * j], hi = P.limit[2 * j + 1];
        gap = std::min(std::fabs(val(theta[j]) - val(lo)), std::fabs(val(theta[j]) - val(hi)));
        if (val(theta[j]) <= val(lo)) {
          r.angA = vneg(ua[j]); r.angB = ua[j];
          r.bias = S(bh) * (theta[j] - lo);
        } else if (val(theta[j]) >= val(hi)) {
          r.angA = ua[j]; r.angB = vneg(ua[j]);
          r.bias = S(bh) * (hi - theta[j]);
        } else {
          r.active = false;
        }
        r.lo = S(0.0);
        break;
      }
      case ORC_MOTOR: {
        int j = sl.idx;
        r.angA = vneg(ua[j]); r.angB = ua[j];
        r.bias = -wstar[j];
        S tmax = P.motor[3 * j + 1] * S(h);
        r.lo = -tmax; r.hi = tmax;
        break;
      }
      case ORC_GN:
      case ORC_GT: {
        int q = sl.idx, a = sl.a;
        V3<S> c = matvec(R[a], get3(P.sph_off, 3 * q));
        V3<S> qc = vadd(p[a], c);
        S rad = P.sph_rad[q];
        S d = qc[2] - rad - S(T.ground_z);
        gap = std::fabs(val(d));
        r.active = val(d) <= 0.0;
        V3<S> ra = vsub(c, vscale(ez, rad));
        if (sl.kind == ORC_GN) {
          r.lin = ez;
          r.angA = cross(ra, ez);
          S vn = dot(r.lin, v[a]) + dot(r.angA, w[a]);
          r.bias = S(bh) * min0(d + S(T.slop)) + P.sph_e[q] * min0(vn);
          r.lo = S(0.0);
        } else {
          V3<S> t1, t2;
          onb(ez, t1, t2);
          r.lin = sl.sub == 0 ? t1 : t2;
          r.angA = cross(ra, r.lin);
          r.friction = true;
          r.mu = P.sph_mu[q];
        }
        break;
      }
      case ORC_PN:
      case ORC_PT: {
        int k = T.pair_sphere[2 * sl.idx], l = T.pair_sphere[2 * sl.idx + 1];
        int a = sl.a, b = sl.b;
        V3<S> ck = matvec(R[a], get3(P.sph_off, 3 * k));
        V3<S> cl = matvec(R[b], get3(P.sph_off, 3 * l));
        V3<S> dlt = vsub(vadd(p[a], ck), vadd(p[b], cl));
        S dist = sqrt(dot(dlt, dlt));
        V3<S> n = val(dist) > 1e-9 ? vscale(dlt, S(1.0) / dist) : ez;
        S d = dist - P.sph_rad[k] - P.sph_rad[l];
        gap = std::fabs(val(d));
        r.active = val(d) <= 0.0;
        V3<S> ra = vsub(ck, vscale(n, P.sph_rad[k]));
        V3<S> rb = vadd(cl, vscale(n, P.sph_rad[l]));
        if (sl.kind == ORC_PN) {
          r.lin = n;
          r.angA = cross(ra, n);
          r.angB = vneg(cross(rb, n));
          S vn = dot(n, vsub(v[a], v[b])) + dot(r.angA, w[a]) + dot(r.angB, w[b]);
          S e = val(P.sph_e[k]) >= val(P.sph_e[l]) ? P.sph_e[k] : P.sph_e[l];
          r.bias = S(bh) * min0(d + S(T.slop)) + e * min0(vn);
          r.lo = S(0.0);
        } else {
          V3<S> t1, t2;
          onb(n, t1, t2);
          r.lin = sl.sub == 0 ? t1 : t2;
          r.angA = cross(ra, r.lin);
          r.angB = vneg(cross(rb, r.lin));
          r.friction = true;
          r.mu = sqrt(P.sph_mu[k] * P.sph_mu[l]);
          if (r.active) gap = std::min(gap, std::fabs(val(n[2])));  // basis sign decision
        }
        break;
      }
    }
    // Effective mass 1 / (J M^-1 J^T + gamma).
    S K = S(0.0);
    if (r.a >= 0) K += invm[r.a] * dot(r.lin, r.lin) + dot(r.angA, matvec(Iinv[r.a], r.angA));
    if (r.b >= 0) K += invm[r.b] * dot(r.lin, r.lin) + dot(r.angB, matvec(Iinv[r.b], r.angB));
    r.meff = S(1.0) / (K + S(T.gamma));
    rows[si] = r;
    if (log) {
      log->active[si] = r.active ? 1 : 0;
      log->gap[si] = gap;
    }
  }

  auto Jv_of = [&](const Row& r) {
    return dot(r.lin, vsub(vof(r.a), vof(r.b))) + dot(r.angA, wvof(r.a)) + dot(r.angB, wvof(r.b));
  };
  auto apply = [&](const Row& r, S dl) {
    if (r.a >= 0) {
      v[r.a] = vadd(v[r.a], vscale(r.lin, dl * invm[r.a]));
      w[r.a] = vadd(w[r.a], vscale(matvec(Iinv[r.a], r.angA), dl));
    }
    if (r.b >= 0) {
      v[r.b] = vsub(v[r.b], vscale(r.lin, dl * invm[r.b]));
      w[r.b] = vadd(w[r.b], vscale(matvec(Iinv[r.b], r.angB), dl));
    }
  };

  // Initial impulses: zero (cold start), or the learned warm start. The warm start works on
  // groups of three rows: the linear rows of a joint, the angular rows of a hinge with its motor
  // row, and the normal and friction rows of a contact. Each group gets 16 features from its
  // assembled rows, the pre-solve velocities and the robot's mass distribution. The start is
  // alpha times the impulses the rows ended the previous step with (lambda_prev) plus each row's
  // effective mass times the network's output for it (a velocity-scale correction, so that an
  // error moves the bodies by about the same speed on stiff and soft rows), projected on the
  // rows' bounds and applied in slot order before the sweeps; a zero network is the damped
  // classic warm start. The network does not see lambda_prev, so it cannot feed the previous
  // impulses back with a gain. The start is a guess, not part of the modelled dynamics: reverse
  // mode treats it as a constant.
  std::vector<S> lam(ns_, S(0.0));
  const std::vector<WsGroup> groups = ws_groups(T, slots);
  auto lp = [&](int si) { return si >= 0 && lam_prev ? lam_prev[si] : 0.0; };
  if (T.warmstart || (log && log->feats)) {
    double mtot = 0.0, pc[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b) {
      const double m = val(P.mass[b]);
      mtot += m;
      for (int k = 0; k < 3; ++k) pc[k] += m * val(p[b][k]);
    }
    for (int k = 0; k < 3; ++k) pc[k] /= mtot;
    int nact = 0;
    for (int si = 0; si < ns_; ++si)
      if ((slots[si].kind == ORC_GN || slots[si].kind == ORC_PN) && rows[si].active) ++nact;
    const double gnorm = std::sqrt(T.gravity[0] * T.gravity[0] + T.gravity[1] * T.gravity[1] + T.gravity[2] * T.gravity[2]);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const WsGroup& G = groups[gi];
      const Slot& s0 = slots[G.slot[0]];
      // the group's point: the contact point on body a, or the joint's anchor on its child body
      V3<S> q;
      if (G.type == WS_GROUND) {
        int qi = s0.idx, a = s0.a;
        q = vadd(p[a], vsub(matvec(R[a], get3(P.sph_off, 3 * qi)), vscale(ez, P.sph_rad[qi])));
      } else if (G.type == WS_PAIR) {
        int k = T.pair_sphere[2 * s0.idx], a = s0.a;
        q = vadd(p[a], vsub(matvec(R[a], get3(P.sph_off, 3 * k)), vscale(rows[G.slot[0]].lin, P.sph_rad[k])));
      } else {
        int j = s0.idx, b = s0.b;
        q = vadd(p[b], matvec(R[b], get3(P.anchor, 6 * j + 3)));
      }
      double phi[ORC_WS_IN];
      for (int k = 0; k < 3; ++k) {
        const int si = G.slot[k];
        const bool on = si >= 0 && rows[si].active;  // rows of inactive slots contribute zeros
        phi[k] = on ? val(Jv_of(rows[si])) : 0.0;
        phi[3 + k] = on ? val(rows[si].bias) : 0.0;
        phi[6 + k] = on ? val(rows[si].meff) : 0.0;
      }
      phi[9] = G.type == WS_GROUND || G.type == WS_PAIR ? val(rows[G.slot[1]].mu)
               : (G.type == WS_HINGE && G.slot[2] >= 0 ? val(rows[G.slot[2]].hi) : 0.0);
      phi[10] = val(q[0]) - pc[0];
      phi[11] = val(q[1]) - pc[1];
      phi[12] = (double)nact;
      phi[13] = mtot * gnorm * h / std::max(1, nact);
      phi[14] = val(q[2]) - T.ground_z;
      phi[15] = (double)G.type;
      if (log && log->feats)
        for (int k = 0; k < ORC_WS_IN; ++k) log->feats[gi * ORC_WS_IN + k] = phi[k];
      if (!T.warmstart) continue;
      double y[ORC_WS_OUT];
      const bool exact_ctrl = g_exact_mlp;  // the warm-start network always keeps its bfloat16 storage
      g_exact_mlp = false;
      ws_forward<double, double>(T.ws_W, phi, y);
      g_exact_mlp = exact_ctrl;
      auto clampd = [](double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); };
      double l0[3] = {0.0, 0.0, 0.0}, z[3];
      for (int k = 0; k < 3; ++k) z[k] = T.ws_alpha * lp(G.slot[k]) + phi[6 + k] * y[k];  // corrected previous impulses
      if (G.type == WS_GROUND || G.type == WS_PAIR) {
        if (rows[G.slot[0]].active) {
          l0[0] = z[0] > 0.0 ? z[0] : 0.0;
          const double hi = val(rows[G.slot[1]].mu) * l0[0];
          l0[1] = clampd(z[1], -hi, hi);
          l0[2] = clampd(z[2], -hi, hi);
        }
      } else {
        for (int k = 0; k < 3; ++k) {
          const int si = G.slot[k];
          if (si < 0 || !rows[si].active) continue;
          l0[k] = slots[si].kind == ORC_MOTOR ? clampd(z[k], val(rows[si].lo), val(rows[si].hi)) : z[k];
        }
      }
      for (int k = 0; k < 3; ++k)
        if (G.slot[k] >= 0) lam[G.slot[k]] = S(l0[k]);
    }
    if (T.warmstart)
      for (int si = 0; si < ns_; ++si)
        if (rows[si].active && val(lam[si]) != 0.0) apply(rows[si], lam[si]);
  }
  if (log && log->lam0)
    for (int si = 0; si < ns_; ++si) log->lam0[si] = val(lam[si]);

  // Projected Gauss-Seidel, fixed number of sweeps in the canonical order:
  // lambda' = clamp(lambda - meff (J v + bias + gamma lambda), lo, hi),
  // then v += M^-1 J^T (lambda' - lambda).
  for (int it = 0; it < T.iters; ++it) {
    for (int oi = 0; oi < ns_; ++oi) {
      int si = order[oi];
      Row& r = rows[si];
      if (!r.active) continue;
      S Jv = Jv_of(r);
      S lo = r.lo, hi = r.hi;
      if (r.friction) {
        hi = r.mu * lam[r.normal];
        lo = -hi;
      }
      S pre = lam[si] - r.meff * (Jv + r.bias + S(T.gamma) * lam[si]);
      S ln = clamp_sel(pre, lo, hi, (int*)nullptr);
      S dl = ln - lam[si];
      lam[si] = ln;
      apply(r, dl);
    }
  }
  if (log && log->lambda)
    for (int si = 0; si < ns_; ++si) log->lambda[si] = val(lam[si]);
  if (lam_out)
    for (int si = 0; si < ns_; ++si) lam_out[si] = val(lam[si]);
  // Residual of the solve: per active row with w = J v + bias + gamma lambda,
  // bilateral |w|; one-sided [0, inf) |min(lambda, w)|; boxed |lambda - clamp(lambda - w, lo, hi)|
  // (motors: +-tau_max h, friction: +-mu lambda_n); RMS over the active rows.
  if (log && log->resid) {
    double ss = 0.0;
    int na = 0;
    for (int si = 0; si < ns_; ++si) {
      const Row& r = rows[si];
      if (!r.active) continue;
      const double wv = val(Jv_of(r)) + val(r.bias) + T.gamma * val(lam[si]), l = val(lam[si]);
      const int kd = slots[si].kind;
      double e;
      if (kd == ORC_JLIN || kd == ORC_JANG) {
        e = wv;
      } else if (kd == ORC_LIMIT || kd == ORC_GN || kd == ORC_PN) {
        e = std::min(l, wv);
      } else {
        double lo = val(r.lo), hi = val(r.hi);
        if (r.friction) { hi = val(r.mu) * val(lam[r.normal]); lo = -hi; }
        double z = l - wv;
        z = z < lo ? lo : (z > hi ? hi : z);
        e = l - z;
      }
      ss += e * e;
      ++na;
    }
    *log->resid = na ? std::sqrt(ss / na) : 0.0;
  }
  if (log && log->bf16_margin) *log->bf16_margin = g_bf16_margin;

  // Semi-implicit Euler with the new velocities, then the Eq. 1 renormalisation.
  xn.resize(x.size());
  for (int b = 0; b < nb; ++b) {
    V3<S> pn = vadd(p[b], vscale(v[b], S(h)));
    M3<S> Wx = {S(0.0), -w[b][2], w[b][1], w[b][2], S(0.0), -w[b][0], -w[b][1], w[b][0], S(0.0)};
    M3<S> WR = matmul(Wx, R[b]);
    M3<S> R1;
    for (int k = 0; k < 9; ++k) R1[k] = R[b][k] + S(h) * WR[k];
    M3<S> RRR = matmul(R1, matmul(transpose(R1), R1));
    for (int k = 0; k < 3; ++k) xn[18 * b + k] = pn[k];
    for (int k = 0; k < 9; ++k) xn[18 * b + 3 + k] = S(0.5) * (S(3.0) * R1[k] - RRR[k]);
    for (int k = 0; k < 3; ++k) xn[18 * b + 12 + k] = v[b][k];
    for (int k = 0; k < 3; ++k) xn[18 * b + 15 + k] = w[b][k];
  }
  if (loss) *loss = w_next != 0.0 ? S(w_next) * loss_of(T, P, xn) : S(0.0);
}

static int check_topo(const orc_topo* T) {
  if (!T || T->nb <= 0 || T->nj < 0 || T->ns < 0 || T->np < 0) return -1;
  for (int j = 0; j < T->nj; ++j) {
    int a = T->joint_body[2 * j], b = T->joint_body[2 * j + 1];
    if (b < 0 || b >= T->nb || a >= T->nb || a == b) return -1;
    if (T->joint_type[j] != ORC_BALL && T->joint_type[j] != ORC_HINGE) return -1;
  }
  for (int q = 0; q < T->ns; ++q)
    if (T->sphere_body[q] < 0 || T->sphere_body[q] >= T->nb) return -1;
  for (int q = 0; q < T->np; ++q) {
    int k = T->pair_sphere[2 * q], l = T->pair_sphere[2 * q + 1];
    if (k < 0 || l < 0 || k >= T->ns || l >= T->ns || T->sphere_body[k] == T->sphere_body[l]) return -1;
  }
  if (T->loss_body < 0 || T->loss_body >= T->nb) return -1;
  if (T->n_recurrent < 0) return -1;
  if (T->n_recurrent > 0 &&
      (T->n_layers < 1 || T->skip || T->widths[0] <= T->n_recurrent || T->widths[T->n_layers] <= T->n_recurrent))
    return -1;
  return 0;
}

template <class S> static Inst<S> lift_inst(const orc_topo& T, const orc_inst& I) {
  Inst<S> P;
  P.mass = lift<S>(I.mass, T.nb);
  P.inertia = lift<S>(I.inertia, 3 * T.nb);
  P.anchor = lift<S>(I.anchor, 6 * T.nj);
  P.axis = lift<S>(I.axis, 6 * T.nj);
  P.ref = lift<S>(I.ref, 6 * T.nj);
  P.limit = lift<S>(I.limit, 2 * T.nj);
  P.motor = lift<S>(I.motor, 3 * T.nj);
  P.sph_off = lift<S>(I.sph_off, 3 * T.ns);
  P.sph_rad = lift<S>(I.sph_rad, T.ns);
  P.sph_mu = lift<S>(I.sph_mu, T.ns);
  P.sph_e = lift<S>(I.sph_e, T.ns);
  P.loss_point = lift<S>(I.loss_point, 3);
  P.loss_target = lift<S>(I.loss_target, 3);
  return P;
}

static double weight_of_state(const orc_topo& T, int t_next, int horizon) {
  if (T.loss_mode == ORC_M_MEAN) return 1.0 / horizon;
  return t_next == horizon ? 1.0 : 0.0;
}

}  // namespace orc

using namespace orc;

extern "C" {

int orc_param_count(int32_t n_layers, const int32_t* widths, int32_t skip) { return param_count(n_layers, widths, skip); }

double orc_bf16(double x) { return bf16(x); }

int orc_num_slots(const orc_topo* T) {
  if (check_topo(T)) return -1;
  return (int)make_slots(*T).size();
}

// Static row schedule: per slot its kind, index, sub-row, bodies, colour; and the sweep order.
int orc_schedule(const orc_topo* T, int32_t* kind, int32_t* idx, int32_t* sub, int32_t* body_a, int32_t* body_b,
                 int32_t* colour, int32_t* order) {
  if (check_topo(T)) return -1;
  auto s = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(s, col, ord);
  for (size_t i = 0; i < s.size(); ++i) {
    kind[i] = s[i].kind; idx[i] = s[i].idx; sub[i] = s[i].sub;
    body_a[i] = s[i].a; body_b[i] = s[i].b;
    colour[i] = col[i]; order[i] = ord[i];
  }
  return (int)s.size();
}

// One step from a given state (used for teacher-forced comparisons), with the solve's residual,
// the warm-start features of every group [orc_ws_groups][16] and the initial impulses [n_slots];
// lam_prev [n_slots] (or NULL: zeros) are the impulses the previous step ended with; h_prev
// [n_recurrent] (or NULL: zeros) the controller's recurrent state, h_next (optional) receives
// the next one.
int orc_step_log(const orc_topo* T, const orc_inst* I, const double* W, int32_t t, const double* x, double* xn,
                 int8_t* active, double* gap, double* lambda, double* bf16_margin, double* resid, double* feats,
                 double* lam0, const double* lam_prev, const double* h_prev, double* h_next) {
  if (check_topo(T)) return -1;
  auto slots = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(slots, col, ord);
  Inst<double> P = lift_inst<double>(*T, *I);
  int np_ = param_count(T->n_layers, T->widths, T->skip);
  std::vector<double> Wv(W ? W : nullptr, W ? W + np_ : nullptr);
  std::vector<double> xs(x, x + 18 * T->nb), xo;
  std::vector<int8_t> act(slots.size());
  std::vector<double> gp(slots.size());
  StepLog lg{active ? active : act.data(), gap ? gap : gp.data(), lambda, bf16_margin, resid, feats, lam0};
  const int H = T->n_recurrent;
  std::vector<double> hin(H, 0.0), hout;
  if (h_prev) std::copy(h_prev, h_prev + H, hin.begin());
  step<double>(*T, slots, ord, P, Wv, t, xs, xo, 0.0, nullptr, &lg, lam_prev, nullptr, &hin, &hout);
  std::memcpy(xn, xo.data(), sizeof(double) * xo.size());
  if (h_next && H > 0) std::memcpy(h_next, hout.data(), sizeof(double) * H);
  return 0;
}

// Mean squared error of the warm-start network over n harvested rows [n][19] (16 features,
// then the 3 converged impulses): loss = (1/n) sum_rows sum_k (y_k - lambda_k)^2, and its
// gradient w.r.t. the ORC_WS_PARAMS parameters (reverse mode, straight-through roundings).
// exact = 1 drops the bfloat16 roundings.
int orc_ws_loss_grad(const double* Wws, const double* rows, int64_t n, int32_t exact, double* loss, double* dW) {
  if (n <= 0) return -1;
  Tape tape;
  Tape* saved = g_tape;
  g_tape = &tape;
  g_exact_mlp = exact != 0;
  double L = 0.0;
  std::vector<double> g(ORC_WS_PARAMS, 0.0);
  for (int64_t r = 0; r < n; ++r) {
    tape.clear();
    std::vector<AD> Wl = lift_leaf(Wws, ORC_WS_PARAMS);
    AD x[ORC_WS_IN], y[ORC_WS_OUT];
    for (int k = 0; k < ORC_WS_IN; ++k) x[k] = AD(rows[r * 19 + k]);
    ws_forward<AD, AD>(Wl.data(), x, y);
    AD e = AD(0.0);
    for (int k = 0; k < ORC_WS_OUT; ++k) {
      AD d = y[k] - AD(rows[r * 19 + ORC_WS_IN + k]);
      e += d * d;
    }
    L += e.v;
    tape.adj.assign(tape.pa.size(), 0.0);
    if (e.id >= 0) tape.adj[e.id] = 1.0;
    tape.backward();
    for (int k = 0; k < ORC_WS_PARAMS; ++k) g[k] += tape.adj[Wl[k].id];
  }
  g_tape = saved;
  g_exact_mlp = false;
  if (loss) *loss = L / (double)n;
  if (dW)
    for (int k = 0; k < ORC_WS_PARAMS; ++k) dW[k] = g[k] / (double)n;
  return 0;
}

// The warm-start network's outputs [n][3] for features [n][16].
int orc_ws_forward(const double* Wws, const double* feats, int64_t n, int32_t exact, double* y) {
  g_exact_mlp = exact != 0;
  for (int64_t r = 0; r < n; ++r) ws_forward<double, double>(Wws, feats + r * ORC_WS_IN, y + r * ORC_WS_OUT);
  g_exact_mlp = false;
  return 0;
}

int orc_ws_param_count() { return ORC_WS_PARAMS; }

// Number of warm-start groups of the topology (rows of the feature log of orc_step_log).
int orc_ws_groups(const orc_topo* T) {
  if (check_topo(T)) return -1;
  return (int)ws_groups(*T, make_slots(*T)).size();
}

// One step from a given state (used for teacher-forced comparisons).
int orc_step(const orc_topo* T, const orc_inst* I, const double* W, int32_t t, const double* x, double* xn,
             int8_t* active, double* gap, double* lambda, double* bf16_margin) {
  if (check_topo(T)) return -1;
  auto slots = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(slots, col, ord);
  Inst<double> P = lift_inst<double>(*T, *I);
  int np_ = param_count(T->n_layers, T->widths, T->skip);
  std::vector<double> Wv(W, W + np_);
  std::vector<double> xs(x, x + 18 * T->nb), xo;
  StepLog lg{active, gap, lambda, bf16_margin};
  step<double>(*T, slots, ord, P, Wv, t, xs, xo, 0.0, nullptr, (active && gap) ? &lg : nullptr);
  std::memcpy(xn, xo.data(), sizeof(double) * xo.size());
  return 0;
}

// Full rollout of `horizon` steps; writes all states [horizon+1][nb][18] (optional), the loss,
// and per step the slot activity / decision distances [horizon][n_slots] (optional).
int orc_rollout_log(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                    double* loss, int8_t* active, double* gap, double* bf16_margin, double* resid);
int orc_rollout(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                double* loss, int8_t* active, double* gap, double* bf16_margin) {
  return orc_rollout_log(T, I, W, horizon, states, loss, active, gap, bf16_margin, nullptr);
}
static int rollout_impl(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                        double* loss, int8_t* active, double* gap, double* bf16_margin, double* resid,
                        std::vector<double>* lam_prevs, double* hs = nullptr);
// Rollout with the controller's recurrent state of every step [horizon + 1][n_recurrent] (h^0 = 0).
int orc_rollout_rec(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                    double* loss, double* hs) {
  return rollout_impl(T, I, W, horizon, states, loss, nullptr, nullptr, nullptr, nullptr, nullptr, hs);
}
// orc_rollout that also gives the residual of every step's solve [horizon].
int orc_rollout_log(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                    double* loss, int8_t* active, double* gap, double* bf16_margin, double* resid) {
  return rollout_impl(T, I, W, horizon, states, loss, active, gap, bf16_margin, resid, nullptr);
}
}  // extern "C"
// The rollout; with the warm start each step starts from the impulses the previous one ended with
// (zero before the first step), and lam_prevs (optional) receives them per step [horizon][n_slots].
static int rollout_impl(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* states,
                        double* loss, int8_t* active, double* gap, double* bf16_margin, double* resid,
                        std::vector<double>* lam_prevs, double* hs) {
  if (check_topo(T) || horizon < 0) return -1;
  auto slots = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(slots, col, ord);
  const int nsl = (int)slots.size();
  Inst<double> P = lift_inst<double>(*T, *I);
  int np_ = param_count(T->n_layers, T->widths, T->skip);
  std::vector<double> Wv(W ? W : nullptr, W ? W + np_ : nullptr);
  std::vector<double> x(I->state0, I->state0 + 18 * T->nb), xn;
  double L = loss_initial(*T, P, x);
  if (states) std::memcpy(states, x.data(), sizeof(double) * x.size());
  std::vector<double> lamp(nsl, 0.0), lamn(nsl, 0.0);
  if (lam_prevs) lam_prevs->assign((size_t)horizon * nsl, 0.0);
  const int H = T->n_recurrent;
  std::vector<double> hcur(H, 0.0), hnext;
  if (hs && H > 0) std::memset(hs, 0, sizeof(double) * H);
  for (int t = 0; t < horizon; ++t) {
    double lt = 0.0;
    std::vector<int8_t> act_tmp;
    std::vector<double> gap_tmp;
    if (resid && !(active && gap)) { act_tmp.resize(nsl); gap_tmp.resize(nsl); }
    StepLog lg{active ? active + (size_t)t * nsl : act_tmp.data(), gap ? gap + (size_t)t * nsl : gap_tmp.data(),
               nullptr, bf16_margin ? bf16_margin + t : nullptr, resid ? resid + t : nullptr, nullptr, nullptr};
    if (lam_prevs) std::copy(lamp.begin(), lamp.end(), lam_prevs->begin() + (size_t)t * nsl);
    step<double>(*T, slots, ord, P, Wv, t, x, xn, weight_of_state(*T, t + 1, horizon), &lt,
                 ((active && gap) || resid) ? &lg : nullptr, T->warmstart ? lamp.data() : nullptr, lamn.data(), &hcur,
                 &hnext);
    lamp.swap(lamn);
    hcur.swap(hnext);
    if (hs && H > 0) std::memcpy(hs + (size_t)(t + 1) * H, hcur.data(), sizeof(double) * H);
    L += lt;
    x.swap(xn);
    if (states) std::memcpy(states + (size_t)(t + 1) * 18 * T->nb, x.data(), sizeof(double) * x.size());
  }
  if (loss) *loss = L;
  return 0;
}
extern "C" {

// Loss and its gradient with respect to the initial state, every per-instance parameter and
// the controller weights: back-propagation through time, one step at a time. Each step is
// replayed on a fresh tape from the stored state x_t with all inputs as leaves, the adjoint
// of x_{t+1} and of the step's loss term are seeded, and the tape is swept backwards.
int orc_rollout_grad(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* loss,
                     const orc_grad* G) {
  if (check_topo(T) || horizon < 1) return -1;
  auto slots = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(slots, col, ord);
  const int nb = T->nb;
  const int np_ = param_count(T->n_layers, T->widths, T->skip);
  std::vector<double> states((size_t)(horizon + 1) * 18 * nb), lamps;
  const int H = T->n_recurrent;
  std::vector<double> hs((size_t)(horizon + 1) * std::max(H, 1));
  if (rollout_impl(T, I, W, horizon, states.data(), loss, nullptr, nullptr, nullptr, nullptr, &lamps, hs.data()))
    return -1;
  const size_t nsl = slots.size();

  Tape tape;
  Tape* saved = g_tape;
  g_tape = &tape;
  auto acc = [](double* dst, const std::vector<AD>& src, const Tape& tp) {
    if (!dst) return;
    for (size_t i = 0; i < src.size(); ++i)
      if (src[i].id >= 0) dst[i] += tp.adj[src[i].id];
  };
  // zero outputs
  auto zero = [](double* d, size_t n) { if (d) std::memset(d, 0, sizeof(double) * n); };
  zero(G->mass, nb); zero(G->inertia, 3 * nb); zero(G->anchor, 6 * T->nj); zero(G->axis, 6 * T->nj);
  zero(G->ref, 6 * T->nj); zero(G->limit, 2 * T->nj); zero(G->motor, 3 * T->nj); zero(G->sph_off, 3 * T->ns);
  zero(G->sph_rad, T->ns); zero(G->sph_mu, T->ns); zero(G->sph_e, T->ns); zero(G->loss_point, 3);
  zero(G->loss_target, 3); zero(G->state0, 18 * nb); zero(G->W, np_);

  std::vector<double> xbar(18 * nb, 0.0), hbar(H, 0.0);
  for (int t = horizon - 1; t >= 0; --t) {
    tape.clear();
    Inst<AD> P;
    P.mass = lift_leaf(I->mass, nb);
    P.inertia = lift_leaf(I->inertia, 3 * nb);
    P.anchor = lift_leaf(I->anchor, 6 * T->nj);
    P.axis = lift_leaf(I->axis, 6 * T->nj);
    P.ref = lift_leaf(I->ref, 6 * T->nj);
    P.limit = lift_leaf(I->limit, 2 * T->nj);
    P.motor = lift_leaf(I->motor, 3 * T->nj);
    P.sph_off = lift_leaf(I->sph_off, 3 * T->ns);
    P.sph_rad = lift_leaf(I->sph_rad, T->ns);
    P.sph_mu = lift_leaf(I->sph_mu, T->ns);
    P.sph_e = lift_leaf(I->sph_e, T->ns);
    P.loss_point = lift_leaf(I->loss_point, 3);
    P.loss_target = lift_leaf(I->loss_target, 3);
    std::vector<AD> Wl = lift_leaf(W, np_);
    std::vector<AD> x = lift_leaf(states.data() + (size_t)t * 18 * nb, 18 * nb), xn;
    std::vector<AD> hin = lift_leaf(hs.data() + (size_t)t * H, H), hout;
    AD lt;
    step<AD>(*T, slots, ord, P, Wl, t, x, xn, weight_of_state(*T, t + 1, horizon), &lt, nullptr,
             T->warmstart ? lamps.data() + (size_t)t * nsl : nullptr, nullptr, &hin, &hout);
    AD l0 = (t == 0) ? loss_initial(*T, P, x) : AD(0.0);
    tape.adj.assign(tape.pa.size(), 0.0);
    // the gradient reaching step t from later steps is decreased by alpha (section 3.2); the
    // loss term of x_{t+1} itself enters undecayed
    const double decay = T->grad_decay > 0.0 ? T->grad_decay : 1.0;
    for (int k = 0; k < 18 * nb; ++k)
      if (xn[k].id >= 0) tape.adj[xn[k].id] += decay * xbar[k];
    for (int k = 0; k < H; ++k)  // the recurrent state's adjoint decays like the state's
      if (hout[k].id >= 0) tape.adj[hout[k].id] += decay * hbar[k];
    if (lt.id >= 0) tape.adj[lt.id] += 1.0;
    if (l0.id >= 0) tape.adj[l0.id] += 1.0;
    tape.backward();
    for (int k = 0; k < 18 * nb; ++k) xbar[k] = x[k].id >= 0 ? tape.adj[x[k].id] : 0.0;
    for (int k = 0; k < H; ++k) hbar[k] = hin[k].id >= 0 ? tape.adj[hin[k].id] : 0.0;
    acc(G->mass, P.mass, tape); acc(G->inertia, P.inertia, tape); acc(G->anchor, P.anchor, tape);
    acc(G->axis, P.axis, tape); acc(G->ref, P.ref, tape); acc(G->limit, P.limit, tape);
    acc(G->motor, P.motor, tape); acc(G->sph_off, P.sph_off, tape); acc(G->sph_rad, P.sph_rad, tape);
    acc(G->sph_mu, P.sph_mu, tape); acc(G->sph_e, P.sph_e, tape); acc(G->loss_point, P.loss_point, tape);
    acc(G->loss_target, P.loss_target, tape); acc(G->W, Wl, tape);
  }
  if (G->state0)
    for (int k = 0; k < 18 * nb; ++k) G->state0[k] += xbar[k];
  g_tape = saved;
  return 0;
}


// Algorithmic work of one instance over `horizon` steps from its initial state: out[0] = forward
// operations per step (counted by the counting scalar), out[1] = reverse-mode operations per
// step (two per recorded partial: one multiply, one add), out[2] = tape nodes per step.
int orc_flops(const orc_topo* T, const orc_inst* I, const double* W, int32_t horizon, double* out) {
  if (check_topo(T) || horizon < 1) return -1;
  auto slots = make_slots(*T);
  std::vector<int> col, ord;
  make_schedule(slots, col, ord);
  const int nb = T->nb;
  const int np_ = param_count(T->n_layers, T->widths, T->skip);
  std::vector<double> states((size_t)(horizon + 1) * 18 * nb);
  if (orc_rollout(T, I, W, horizon, states.data(), nullptr, nullptr, nullptr, nullptr)) return -1;
  Inst<CNT> Pc = lift_inst<CNT>(*T, *I);
  std::vector<CNT> Wc(np_);
  for (int k = 0; k < np_; ++k) Wc[k] = CNT(W[k]);
  double fwd = 0.0, rev = 0.0, nodes = 0.0;
  Tape tape;
  Tape* saved = g_tape;
  g_tape = &tape;
  for (int t = 0; t < horizon; ++t) {
    std::vector<CNT> x(18 * nb), xn;
    for (int k = 0; k < 18 * nb; ++k) x[k] = CNT(states[(size_t)t * 18 * nb + k]);
    CNT lt;
    double f0 = g_flops;
    step<CNT>(*T, slots, ord, Pc, Wc, t, x, xn, weight_of_state(*T, t + 1, horizon), &lt, nullptr);
    fwd += g_flops - f0;
    tape.clear();
    Inst<AD> P;
    P.mass = lift_leaf(I->mass, nb); P.inertia = lift_leaf(I->inertia, 3 * nb);
    P.anchor = lift_leaf(I->anchor, 6 * T->nj); P.axis = lift<AD>(I->axis, 6 * T->nj);
    P.ref = lift<AD>(I->ref, 6 * T->nj); P.limit = lift_leaf(I->limit, 2 * T->nj);
    P.motor = lift_leaf(I->motor, 3 * T->nj); P.sph_off = lift_leaf(I->sph_off, 3 * T->ns);
    P.sph_rad = lift_leaf(I->sph_rad, T->ns); P.sph_mu = lift_leaf(I->sph_mu, T->ns);
    P.sph_e = lift_leaf(I->sph_e, T->ns); P.loss_point = lift_leaf(I->loss_point, 3);
    P.loss_target = lift_leaf(I->loss_target, 3);
    std::vector<AD> Wl = lift_leaf(W, np_);
    std::vector<AD> xa = lift_leaf(states.data() + (size_t)t * 18 * nb, 18 * nb), xna;
    AD la;
    size_t n0 = tape.pa.size();
    step<AD>(*T, slots, ord, P, Wl, t, xa, xna, weight_of_state(*T, t + 1, horizon), &la, nullptr);
    for (size_t q = n0; q < tape.pa.size(); ++q) {
      rev += 2.0 * ((tape.pa[q] >= 0) + (tape.pb[q] >= 0));
      nodes += 1.0;
    }
  }
  g_tape = saved;
  out[0] = fwd / horizon;
  out[1] = rev / horizon;
  out[2] = nodes / horizon;
  return 0;
}

}  // extern "C"

// ========================================================================================
// Differentiable camera (section 3.4, the inverted pendulum seen by a camera): a pinhole ray
// tracer over textured oriented boxes carried by the bodies. Per pixel (row i, column j) the ray
// from the camera centre C runs along d = R_c^T (P ((j + 1/2) - W/2) / f, P ((i + 1/2) - H/2) / f, P)
// (f: focal length in pixels, P: distance of the projection plane), so that t = 1 is the
// projection plane; every box is intersected (slab test in the box's frame), and of
// the hits at t >= 1 (in front of the projection plane) the nearest is kept. The hit face (the
// box axis k of the entry slab) gives texture coordinates from the two other local coordinates,
// u = (x_a / h_a + 1) / 2, v = (x_b / h_b + 1) / 2 with a = (k + 1) mod 3, b = (k + 2) mod 3,
// and the colour is the bilinear interpolation of the box's texture (texel centres at
// ((c + 1/2) / Wt, (r + 1/2) / Ht), clamped at the edges), which gives the frame non-zero
// derivatives with respect to the state and the texture. Rays that hit nothing are black.
// Spheres (kind 1, radius = half[0]) are intersected as |C + t d - c_w| = r; their texture
// coordinates come from the hit point's direction in the sphere's body frame,
// u = atan2(y, x) / (2 pi) + 1/2, v = acos(z / r) / pi. A plane (kind 2) is the plane z = 0 of
// the object's frame (a ground plane, seen from either side); its texture repeats with periods
// 2 half[0] and 2 half[1] along the frame's x and y: u = frac(x / (2 half[0]) + 1/2),
// v = frac(y / (2 half[1]) + 1/2).
// Reverse mode keeps the discrete choices (which object, which face, which texels) of the forward
// pass and differentiates the rest (the oracle's tape).
extern "C" {
typedef struct {
  int32_t W, H;     // image width and height in pixels
  double f;         // focal length in pixels
  double plane;     // distance of the projection plane from C (world units); hits before it are not seen
  double pos[3];    // camera centre C (world)
  double rot[9];    // R_c, row-major: rows are the camera's x (image right), y (image down) and z (optical) axes
} orc_camera;
typedef struct {
  int32_t n_obj;
  const int32_t* body;    // [n_obj] body carrying the box (-1: the world)
  const double* center;   // [n_obj][3] box centre in the body frame
  const double* half;     // [n_obj][3] half extents along the body axes
  const int32_t* tex;     // [n_obj] texture index
  int32_t n_tex, tex_h, tex_w;
  const double* tex_data; // [n_tex][tex_h][tex_w][3]
  const int32_t* kind;    // [n_obj] 0 = box, 1 = sphere of radius half[0], 2 = plane (NULL: all boxes)
} orc_scene;
}  // extern "C"

namespace orc {

template <class S>
static void render_impl(const orc_camera& cam, const orc_scene& sc, const std::vector<S>& x, const std::vector<S>& tex,
                        std::vector<S>& img, int32_t* hit_obj) {
  const int W = cam.W, H = cam.H, th = sc.tex_h, tw = sc.tex_w;
  img.assign((size_t)W * H * 3, S(0.0));
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      const double dc[3] = {cam.plane * ((j + 0.5) - 0.5 * W) / cam.f, cam.plane * ((i + 0.5) - 0.5 * H) / cam.f, cam.plane};
      double d[3];
      for (int r = 0; r < 3; ++r) d[r] = cam.rot[0 * 3 + r] * dc[0] + cam.rot[1 * 3 + r] * dc[1] + cam.rot[2 * 3 + r] * dc[2];
      int best = -1, bk = 0;
      double bt = INFINITY;
      S bl[3], dl[3];  // ray in the best box's frame
      for (int o = 0; o < sc.n_obj; ++o) {
        const int b = sc.body[o];
        // box frame: centre c_w = p + R c, axes = columns of R (R maps body to world)
        S R[9], p[3];
        for (int k = 0; k < 9; ++k) R[k] = b >= 0 ? x[18 * b + 3 + k] : S(k % 4 == 0 ? 1.0 : 0.0);
        for (int k = 0; k < 3; ++k) p[k] = b >= 0 ? x[18 * b + k] : S(0.0);
        S cw[3], ol[3], dlo[3];
        for (int r = 0; r < 3; ++r)
          cw[r] = p[r] + R[3 * r] * sc.center[3 * o] + R[3 * r + 1] * sc.center[3 * o + 1] + R[3 * r + 2] * sc.center[3 * o + 2];
        for (int k = 0; k < 3; ++k) {  // R^T (C - c_w), R^T d
          ol[k] = R[k] * (S(cam.pos[0]) - cw[0]) + R[3 + k] * (S(cam.pos[1]) - cw[1]) + R[6 + k] * (S(cam.pos[2]) - cw[2]);
          dlo[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];
        }
        if (sc.kind && sc.kind[o] == 2) {  // plane z = 0 of the object frame
          if (val(dlo[2]) == 0.0) continue;
          const double tn = -val(ol[2]) / val(dlo[2]);
          if (!(tn >= 1.0) || !(tn < bt)) continue;
          best = o; bk = -2; bt = tn;
          for (int k = 0; k < 3; ++k) { bl[k] = ol[k]; dl[k] = dlo[k]; }
          continue;
        }
        if (sc.kind && sc.kind[o] == 1) {  // sphere: a t^2 + 2 b t + c = 0 in the body frame
          const double r = sc.half[3 * o];
          const double a = val(dlo[0]) * val(dlo[0]) + val(dlo[1]) * val(dlo[1]) + val(dlo[2]) * val(dlo[2]);
          const double b = val(dlo[0]) * val(ol[0]) + val(dlo[1]) * val(ol[1]) + val(dlo[2]) * val(ol[2]);
          const double c = val(ol[0]) * val(ol[0]) + val(ol[1]) * val(ol[1]) + val(ol[2]) * val(ol[2]) - r * r;
          const double disc = b * b - a * c;
          if (!(disc >= 0.0)) continue;
          const double tn = (-b - std::sqrt(disc)) / a;
          if (!(tn >= 1.0) || !(tn < bt)) continue;
          best = o; bk = -1; bt = tn;
          for (int k = 0; k < 3; ++k) { bl[k] = ol[k]; dl[k] = dlo[k]; }
          continue;
        }
        double tn = -INFINITY, tf = INFINITY;
        int kn = 0;
        bool miss = false;
        for (int k = 0; k < 3; ++k) {
          const double h = sc.half[3 * o + k];
          if (val(dlo[k]) == 0.0) {
            if (std::fabs(val(ol[k])) > h) miss = true;
            continue;
          }
          double t1 = (-h - val(ol[k])) / val(dlo[k]), t2 = (h - val(ol[k])) / val(dlo[k]);
          if (t1 > t2) std::swap(t1, t2);
          if (t1 > tn) { tn = t1; kn = k; }
          tf = std::min(tf, t2);
        }
        if (miss || !(tn <= tf) || !(tn >= 1.0) || !(tn < bt)) continue;
        best = o; bk = kn; bt = tn;
        for (int k = 0; k < 3; ++k) { bl[k] = ol[k]; dl[k] = dlo[k]; }
      }
      if (hit_obj) hit_obj[(size_t)i * W + j] = best;
      if (best < 0) continue;
      S u, v;
      if (bk == -2) {  // plane: in-plane coordinates of the hit point, the texture repeated
        S t = -bl[2] / dl[2];
        S uu = (bl[0] + t * dl[0]) / S(2.0 * sc.half[3 * best]) + S(0.5);
        S vv = (bl[1] + t * dl[1]) / S(2.0 * sc.half[3 * best + 1]) + S(0.5);
        u = uu - S(std::floor(val(uu)));
        v = vv - S(std::floor(val(vv)));
      } else if (bk < 0) {  // sphere: the near root, then the hit direction's spherical angles
        const double r = sc.half[3 * best];
        S a = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
        S b = dl[0] * bl[0] + dl[1] * bl[1] + dl[2] * bl[2];
        S c = bl[0] * bl[0] + bl[1] * bl[1] + bl[2] * bl[2] - S(r * r);
        S t = (-b - sqrt(b * b - a * c)) / a;
        S px = bl[0] + t * dl[0], py = bl[1] + t * dl[1], pz = bl[2] + t * dl[2];
        u = atan2(py, px) / S(2.0 * M_PI) + S(0.5);
        double zr = val(pz) / r;
        zr = zr > 1.0 ? 1.0 : (zr < -1.0 ? -1.0 : zr);
        // v = acos(pz / r) / pi, d v / d pz = -1 / (pi r sqrt(1 - (pz/r)^2))
        const double vv = std::acos(zr) / M_PI;
        const double dv = -1.0 / (M_PI * r * std::sqrt(std::max(1e-300, 1.0 - zr * zr)));
        v = S(vv) + (pz - S(val(pz))) * S(dv);
      } else {
        // the entry plane: x_k = s h_k with s = -sign(d_k)
        const double hk = sc.half[3 * best + bk];
        const double s = val(dl[bk]) > 0.0 ? -1.0 : 1.0;
        S t = (S(s * hk) - bl[bk]) / dl[bk];
        const int a = (bk + 1) % 3, c = (bk + 2) % 3;
        u = ((bl[a] + t * dl[a]) / S(sc.half[3 * best + a]) + S(1.0)) * S(0.5);
        v = ((bl[c] + t * dl[c]) / S(sc.half[3 * best + c]) + S(1.0)) * S(0.5);
      }
      // bilinear texture sample, texel centres at (c + 1/2) / tw, clamped at the edges
      S xs = u * S((double)tw) - S(0.5), ys = v * S((double)th) - S(0.5);
      const double x0f = std::floor(val(xs)), y0f = std::floor(val(ys));
      S fx = xs - S(x0f), fy = ys - S(y0f);
      auto cl = [](int q, int n) { return q < 0 ? 0 : (q >= n ? n - 1 : q); };
      const int x0 = cl((int)x0f, tw), x1 = cl((int)x0f + 1, tw), y0 = cl((int)y0f, th), y1 = cl((int)y0f + 1, th);
      const size_t tb = (size_t)sc.tex[best] * th * tw * 3;
      for (int ch = 0; ch < 3; ++ch) {
        const S t00 = tex[tb + ((size_t)y0 * tw + x0) * 3 + ch], t01 = tex[tb + ((size_t)y0 * tw + x1) * 3 + ch];
        const S t10 = tex[tb + ((size_t)y1 * tw + x0) * 3 + ch], t11 = tex[tb + ((size_t)y1 * tw + x1) * 3 + ch];
        img[((size_t)i * W + j) * 3 + ch] = (S(1.0) - fy) * ((S(1.0) - fx) * t00 + fx * t01) + fy * ((S(1.0) - fx) * t10 + fx * t11);
      }
    }
}

}  // namespace orc

extern "C" {

// Frame [H][W][3] of the scene for one instance's state [nb][18]; hit_obj [H][W] (optional)
// receives the index of the box each pixel sees (-1: none).
int orc_render(const orc_camera* cam, const orc_scene* sc, int32_t nb, const double* state, double* image,
               int32_t* hit_obj) {
  if (!cam || !sc || cam->W < 1 || cam->H < 1 || sc->tex_h < 1 || sc->tex_w < 1) return -1;
  std::vector<double> x(state, state + 18 * nb), tex(sc->tex_data, sc->tex_data + (size_t)sc->n_tex * sc->tex_h * sc->tex_w * 3), img;
  render_impl<double>(*cam, *sc, x, tex, img, hit_obj);
  std::memcpy(image, img.data(), sizeof(double) * img.size());
  return 0;
}

// Reverse mode of orc_render for the scalar sum(dimage * image): its gradient with respect to
// the state [nb][18] (dstate; velocities get zero) and to every texel (dtex, optional).
int orc_render_grad(const orc_camera* cam, const orc_scene* sc, int32_t nb, const double* state, const double* dimage,
                    double* dstate, double* dtex) {
  if (!cam || !sc || cam->W < 1 || cam->H < 1 || sc->tex_h < 1 || sc->tex_w < 1) return -1;
  Tape tape;
  Tape* saved = g_tape;
  g_tape = &tape;
  const size_t ntex = (size_t)sc->n_tex * sc->tex_h * sc->tex_w * 3;
  std::vector<AD> x = lift_leaf(state, 18 * nb), tex = lift_leaf(sc->tex_data, ntex), img;
  render_impl<AD>(*cam, *sc, x, tex, img, nullptr);
  tape.adj.assign(tape.pa.size(), 0.0);
  for (size_t k = 0; k < img.size(); ++k)
    if (img[k].id >= 0) tape.adj[img[k].id] += dimage[k];
  tape.backward();
  for (int k = 0; k < 18 * nb; ++k) dstate[k] = tape.adj[x[k].id];
  if (dtex)
    for (size_t k = 0; k < ntex; ++k) dtex[k] = tape.adj[tex[k].id];
  g_tape = saved;
  return 0;
}

}  // extern "C"
