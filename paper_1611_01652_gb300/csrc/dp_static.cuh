// Compile-time specialisation of the projected Gauss-Seidel sweeps (forward and reverse) for
// robot topologies known when the library is built. The slot schedule is computed by constexpr
// code from the same rules as the run-time path (canonical slot order, greedy colouring,
// colour-major sweep), so slot kinds, bodies and the sweep order are constants: the row loop is
// fully unrolled, body velocities and impulses live in registers and every shared-memory row
// field is read at a constant offset. A world whose topology matches one of these uses them;
// any other topology uses the run-time loops.
#pragma once
#include <utility>

#include "dp_adjoint.cuh"

extern __shared__ float g_smem[];

struct TopoDesc {
  int nb, nj, ns, np;
  int jtype[DPK_MAXJ], ja[DPK_MAXJ], jb[DPK_MAXJ], jflags[DPK_MAXJ];
  int sbody[DPK_MAXS], pk[DPK_MAXP], pl[DPK_MAXP];
};

struct SlotTab {
  int n;
  int kind[DPK_MAXSLOT], idx[DPK_MAXSLOT], sub[DPK_MAXSLOT], a[DPK_MAXSLOT], b[DPK_MAXSLOT], normal[DPK_MAXSLOT],
      colour[DPK_MAXSLOT], order[DPK_MAXSLOT];
};

constexpr void slot_push(SlotTab& S, int kind, int idx, int sub, int a, int b, int normal) {
  S.kind[S.n] = kind; S.idx[S.n] = idx; S.sub[S.n] = sub; S.a[S.n] = a; S.b[S.n] = b; S.normal[S.n] = normal;
  ++S.n;
}

constexpr SlotTab build_schedule(const TopoDesc& d) {
  SlotTab S{};
  for (int j = 0; j < d.nj; ++j) {
    for (int k = 0; k < 3; ++k) slot_push(S, RK_JLIN, j, k, d.ja[j], d.jb[j], -1);
    if (d.jtype[j] == 1)
      for (int k = 0; k < 2; ++k) slot_push(S, RK_JANG, j, k, d.ja[j], d.jb[j], -1);
  }
  for (int j = 0; j < d.nj; ++j)
    if (d.jtype[j] == 1 && (d.jflags[j] & 1)) slot_push(S, RK_LIMIT, j, 0, d.ja[j], d.jb[j], -1);
  for (int j = 0; j < d.nj; ++j)
    if (d.jtype[j] == 1 && (d.jflags[j] & 2)) slot_push(S, RK_MOTOR, j, 0, d.ja[j], d.jb[j], -1);
  for (int q = 0; q < d.ns; ++q) {
    const int n = S.n;
    slot_push(S, RK_GN, q, 0, d.sbody[q], -1, -1);
    slot_push(S, RK_GT, q, 0, d.sbody[q], -1, n);
    slot_push(S, RK_GT, q, 1, d.sbody[q], -1, n);
  }
  for (int q = 0; q < d.np; ++q) {
    const int n = S.n;
    const int a = d.sbody[d.pk[q]], b = d.sbody[d.pl[q]];
    slot_push(S, RK_PN, q, 0, a, b, -1);
    slot_push(S, RK_PT, q, 0, a, b, n);
    slot_push(S, RK_PT, q, 1, a, b, n);
  }
  for (int i = 0; i < S.n; ++i) {
    bool used[DPK_MAXSLOT + 1] = {};
    for (int k = 0; k < i; ++k) {
      const bool share = (S.a[i] >= 0 && (S.a[i] == S.a[k] || S.a[i] == S.b[k])) ||
                         (S.b[i] >= 0 && (S.b[i] == S.a[k] || S.b[i] == S.b[k]));
      if (share) used[S.colour[k]] = true;
    }
    int c = 0;
    while (used[c]) ++c;
    S.colour[i] = c;
  }
  // stable sort of slot indices by colour (insertion sort)
  for (int i = 0; i < S.n; ++i) S.order[i] = i;
  for (int i = 1; i < S.n; ++i) {
    const int x = S.order[i];
    int j = i - 1;
    while (j >= 0 && S.colour[S.order[j]] > S.colour[x]) {
      S.order[j + 1] = S.order[j];
      --j;
    }
    S.order[j + 1] = x;
  }
  return S;
}

// The quadruped of the benchmark: torso (body 0), legs l = 0..3 with an upper link 1+2l on a
// hip hinge and a lower link 2+2l on a knee hinge, both with limit and servo; a foot sphere on
// each lower link and four spheres inside the torso.
struct QuadrupedTopo {
  static constexpr TopoDesc desc = {
      9, 8, 8, 0,
      {1, 1, 1, 1, 1, 1, 1, 1},
      {0, 1, 0, 3, 0, 5, 0, 7},
      {1, 2, 3, 4, 5, 6, 7, 8},
      {3, 3, 3, 3, 3, 3, 3, 3},
      {2, 4, 6, 8, 0, 0, 0, 0},
      {},
      {}};
  static constexpr SlotTab S = build_schedule(desc);
  static constexpr int NB = desc.nb;
  static constexpr int NS = S.n;
  static constexpr int id = 1;
  static constexpr int CTRL_H = 128;  // hidden width of the tensor-core controller its kernels carry
};

// The robot arms of the uneven batch: N links on hinges stacked from the world (joint 0 yaws with
// a servo only, joints 1 .. N-1 pitch with limits and servos) and a sphere on the last link; their
// controller is the 256-wide tensor-core network.
template <int N>
struct ArmTopo {
  static constexpr TopoDesc make() {
    TopoDesc d{};
    d.nb = N;
    d.nj = N;
    d.ns = 1;
    d.np = 0;
    for (int j = 0; j < N; ++j) {
      d.jtype[j] = 1;
      d.ja[j] = j - 1;
      d.jb[j] = j;
      d.jflags[j] = j == 0 ? 2 : 3;
    }
    d.sbody[0] = N - 1;
    return d;
  }
  static constexpr TopoDesc desc = make();
  static constexpr SlotTab S = build_schedule(desc);
  static constexpr int NB = N;
  static constexpr int NS = S.n;
  static constexpr int id = 10 + N;
  static constexpr int CTRL_H = 256;
};

// Host-side check: does the descriptor's topology equal a compiled one? Returns its id or 0.
template <class Q>
inline bool topo_matches(int nb, int nj, int ns, int np, const int* jtype, const int* jbody, const int* jflags,
                         const int* sbody, const int* pair) {
  const TopoDesc& d = Q::desc;
  if (nb != d.nb || nj != d.nj || ns != d.ns || np != d.np) return false;
  for (int j = 0; j < nj; ++j)
    if (jtype[j] != d.jtype[j] || jbody[2 * j] != d.ja[j] || jbody[2 * j + 1] != d.jb[j] || jflags[j] != d.jflags[j])
      return false;
  for (int q = 0; q < ns; ++q)
    if (sbody[q] != d.sbody[q]) return false;
  for (int q = 0; q < np; ++q)
    if (pair[2 * q] != d.pk[q] || pair[2 * q + 1] != d.pl[q]) return false;
  return true;
}

// ---------------------------------------------------------------------------- helpers
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int KIND, int SUB>
__device__ __forceinline__ constexpr bool lin_is_constant() {
  return KIND == RK_JLIN || KIND == RK_GN || KIND == RK_GT;
}
template <int KIND, int SUB>
__device__ __forceinline__ float3 const_lin() {
  if (KIND == RK_JLIN) return f3(SUB == 0 ? 1.f : 0.f, SUB == 1 ? 1.f : 0.f, SUB == 2 ? 1.f : 0.f);
  if (KIND == RK_GN) return f3(0.f, 0.f, 1.f);
  if (KIND == RK_GT) return f3(SUB == 0 ? 1.f : 0.f, SUB == 1 ? 1.f : 0.f, 0.f);
  return f3(0.f, 0.f, 0.f);
}
// The axis (0, 1, 2) of a constant linear Jacobian part that is a unit vector, -1 for rows
// without a linear part, -2 when it is not a compile-time constant (sphere pairs). Products with
// the part's zero components add exact zeros, which IEEE arithmetic does not let the compiler
// drop (0 * x is not 0 for infinite or NaN x): the sweeps skip them. The sums are the same up to
// where the compiler fuses a product into an add.
template <int KIND, int SUB>
__device__ __forceinline__ constexpr int lin_axis() {
  if (KIND == RK_JLIN || KIND == RK_GT) return SUB;
  if (KIND == RK_GN) return 2;
  if (KIND == RK_JANG || KIND == RK_LIMIT || KIND == RK_MOTOR) return -1;
  return -2;
}
template <int KIND>
__device__ __forceinline__ constexpr bool lin_is_zero() {
  return KIND == RK_JANG || KIND == RK_LIMIT || KIND == RK_MOTOR;
}
template <int KIND>
__device__ __forceinline__ constexpr bool maybe_inactive() {
  return KIND == RK_LIMIT || KIND >= RK_GN;
}

// ---------------------------------------------------------------------------- forward sweeps
template <class Q, bool TAPE, class RV>
__device__ void pgs_solve_static(const DevTopo& T, const LaneT<RV>& L, const SL& X, const TapeStep& tp) {
  constexpr int NB = Q::NB, NS = Q::NS;
  const SL& S = L.S;
  float v[NB][6], im[NB], lam[NS];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[b][k] = X[18 * b + 12 + k];
    im[b] = S[T.sm_invm + b];
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) lam[s] = T.ws ? S[T.sm_lam + s] : 0.f;
  const float gamma = T.gamma;
  for (int it = 0; it < T.iters; ++it) {
    static_for<NS>([&](auto OI) {
      constexpr int s = Q::S.order[decltype(OI)::value];
      constexpr int kind = Q::S.kind[s], sub = Q::S.sub[s], a = Q::S.a[s], b = Q::S.b[s];
      const RV R = L.rows.at(s * RF_N);
      const float meff = R[RF_MEFF];
      if (maybe_inactive<kind>() && !__any_sync(FULLMASK, meff != 0.f)) return;
      constexpr int ax = lin_axis<kind, sub>();
      float3 lin = f3(0.f, 0.f, 0.f);
      if constexpr (ax == -2) lin = R.v3(RF_LIN);
      float Jv = 0.f;
      float3 angA = f3(0.f, 0.f, 0.f), angB = angA;
      if (a >= 0) {
        angA = R.v3(RF_ANGA);
        if constexpr (ax >= 0)
          Jv += v[a][ax] + angA.x * v[a][3] + angA.y * v[a][4] + angA.z * v[a][5];
        else if constexpr (ax == -1)
          Jv += angA.x * v[a][3] + angA.y * v[a][4] + angA.z * v[a][5];
        else
          Jv += lin.x * v[a][0] + lin.y * v[a][1] + lin.z * v[a][2] + angA.x * v[a][3] + angA.y * v[a][4] + angA.z * v[a][5];
      }
      if (b >= 0) {
        angB = R.v3(RF_ANGB);
        if constexpr (ax >= 0)
          Jv += angB.x * v[b][3] + angB.y * v[b][4] + angB.z * v[b][5] - v[b][ax];
        else if constexpr (ax == -1)
          Jv += angB.x * v[b][3] + angB.y * v[b][4] + angB.z * v[b][5];
        else
          Jv += angB.x * v[b][3] + angB.y * v[b][4] + angB.z * v[b][5] - (lin.x * v[b][0] + lin.y * v[b][1] + lin.z * v[b][2]);
      }
      const float l0 = lam[s];
      const float pre = l0 - meff * (Jv + R[RF_BIAS] + gamma * l0);
      float lo, hi;
      if constexpr (kind == RK_GT || kind == RK_PT) {
        constexpr int nrm = Q::S.normal[s];
        hi = R[RF_BND] * lam[nrm];
        lo = -hi;
      } else if constexpr (kind == RK_MOTOR) {
        hi = R[RF_BND];
        lo = -hi;
      } else if constexpr (kind == RK_JLIN || kind == RK_JANG) {
        lo = -__int_as_float(0x7f800000);
        hi = __int_as_float(0x7f800000);
      } else {
        lo = 0.f;
        hi = __int_as_float(0x7f800000);
      }
      const int br = pre < lo ? 1 : (pre > hi ? 2 : 0);
      const float ln = br == 1 ? lo : (br == 2 ? hi : pre);
      const float dl = ln - l0;
      lam[s] = ln;
      if (a >= 0) {
        const float c = dl * im[a];
        const float3 IA = R.v3(RF_IA);
        if constexpr (ax >= 0) {
          v[a][ax] += c;
        } else if constexpr (ax == -2) {
          v[a][0] += c * lin.x; v[a][1] += c * lin.y; v[a][2] += c * lin.z;
        }
        v[a][3] += dl * IA.x; v[a][4] += dl * IA.y; v[a][5] += dl * IA.z;
      }
      if (b >= 0) {
        const float c = dl * im[b];
        const float3 IB = R.v3(RF_IB);
        if constexpr (ax >= 0) {
          v[b][ax] -= c;
        } else if constexpr (ax == -2) {
          v[b][0] -= c * lin.x; v[b][1] -= c * lin.y; v[b][2] -= c * lin.z;
        }
        v[b][3] += dl * IB.x; v[b][4] += dl * IB.y; v[b][5] += dl * IB.z;
      }
      if (TAPE) {
        const int o = (it * NS + s) * 32;
        tp.lam[o] = ln;
        tp.br[o] = (uint8_t)br;
      }
    });
    if (TAPE) {
      float* vi = tp.viter + it * NB * 6 * 32;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < 6; ++k) vi[(6 * b + k) * 32] = v[b][k];
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int k = 0; k < 6; ++k) X[18 * b + 12 + k] = v[b][k];
#pragma unroll
  for (int s = 0; s < NS; ++s) S[T.sm_lam + s] = lam[s];
}

// ---------------------------------------------------------------------------- reverse sweeps
// Same arithmetic as pgs_reverse with constant slots. Working velocities live in registers;
// velocity adjoints, impulse adjoints and row-adjoint accumulators in shared memory; I^-1 J^T is
// recomputed from the on-chip world inverse inertias. Which rows are active on some lane is
// decided once per step (a bit mask), and the clamp branch enters the arithmetic as a selector.
// Every tape value a row needs (row fields, its impulse before and after the sweep, the clamp
// branch, the contact's normal impulse) is loaded one row ahead of its use, so the L2 latency of
// the tape overlaps the arithmetic of the row before (the last row of a sweep prefetches the
// first row of the sweep before it).
// Called with a read-only tape view (the whole tape was recorded by the rollout kernel).
struct RowIn {
  float meff, bias, la, lb, bnd, lnrm;
  float3 lin, angA, angB;
  int br;
};

// Position of slot s in the sweep order.
template <class Q>
__device__ __forceinline__ constexpr int order_pos(int s) {
  for (int k = 0; k < Q::NS; ++k)
    if (Q::S.order[k] == s) return k;
  return -1;
}

template <class Q, int s>
__device__ __forceinline__ RowIn load_row(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it) {
  constexpr int NS = Q::NS;
  constexpr int kind = Q::S.kind[s], sub = Q::S.sub[s], a = Q::S.a[s], b = Q::S.b[s];
  const GSR R = L.rows.at(s * RF_N);
  RowIn r;
  r.meff = R[RF_MEFF];
  r.bias = R[RF_BIAS];
  if constexpr (lin_is_constant<kind, sub>()) r.lin = const_lin<kind, sub>();
  else if constexpr (lin_is_zero<kind>()) r.lin = f3(0.f, 0.f, 0.f);
  else r.lin = R.v3(RF_LIN);
  r.angA = a >= 0 ? R.v3(RF_ANGA) : f3(0.f, 0.f, 0.f);
  r.angB = b >= 0 ? R.v3(RF_ANGB) : f3(0.f, 0.f, 0.f);
  const int o = (it * NS + s) * 32;
  r.la = __ldg(tp.lam + o);
  r.lb = it > 0 ? __ldg(tp.lam + o - NS * 32) : (T.ws ? __ldg(tp.lam0 + s * 32) : 0.f);
  r.br = __ldg(tp.br + o);
  r.bnd = 0.f;
  r.lnrm = 0.f;
  if constexpr (kind == RK_GT || kind == RK_PT) {
    // the contact's normal impulse as the friction row saw it: after this sweep when the normal
    // row comes first in the sweep order, else before it
    constexpr int nrm = Q::S.normal[s];
    r.bnd = R[RF_BND];
    if constexpr (order_pos<Q>(nrm) < order_pos<Q>(s))
      r.lnrm = __ldg(tp.lam + (it * NS + nrm) * 32);
    else
      r.lnrm = it > 0 ? __ldg(tp.lam + ((it - 1) * NS + nrm) * 32) : (T.ws ? __ldg(tp.lam0 + nrm * 32) : 0.f);
  }
  return r;
}

template <class Q>
__device__ __noinline__ void pgs_reverse_static(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp) {
  constexpr int NB = Q::NB, NS = Q::NS;
  constexpr int NW = (NS + 31) / 32;
  // shared-memory views re-derived from the __shared__ array so their address space is known
  const SL S{g_smem + (threadIdx.x & 31)};
  const SL VB = S.at(T.sm_vb), RC = S.at(T.sm_rc);
  const float gamma = T.gamma;
  const int iters = T.iters;
  // v: working velocities; ib9r, imbr: adjoints of the world inverse inertias and inverse
  // masses, summed in registers over the sweeps (added to their zeroed shared-memory
  // accumulators at the end, so the sums are the same)
  float v[NB][6], im[NB], ib9r[NB][9], imbr[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    im[b] = S[T.sm_invm + b];
    imbr[b] = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) ib9r[b][k] = 0.f;
  }
  unsigned live[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) live[w] = 0u;
  static_for<NS>([&](auto SI) {
    constexpr int s = decltype(SI)::value;
    if constexpr (maybe_inactive<Q::S.kind[s]>()) {
      const float meff = L.rows.at(s * RF_N)[RF_MEFF];
      if (__any_sync(FULLMASK, meff != 0.f)) live[s >> 5] |= 1u << (s & 31);
    } else {
      live[s >> 5] |= 1u << (s & 31);
    }
  });
#pragma unroll
  for (int s = 0; s < NS; ++s) S[T.sm_lam + s] = 0.f;
  RowIn cur = load_row<Q, Q::S.order[NS - 1]>(T, L, tp, iters - 1);
  for (int it = iters - 1; it >= 0; --it) {
    {
      const float* vi = tp.viter + it * NB * 6 * 32;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[b][k] = __ldg(vi + (6 * b + k) * 32);
    }
    static_for<NS>([&](auto RI) {
      constexpr int ri = decltype(RI)::value;
      constexpr int s = Q::S.order[NS - 1 - ri];
      constexpr int kind = Q::S.kind[s], a = Q::S.a[s], b = Q::S.b[s];
      RowIn nxt;
      if constexpr (ri + 1 < NS) {
        nxt = load_row<Q, Q::S.order[NS - 2 - ri]>(T, L, tp, it);
      } else {
        nxt = it > 0 ? load_row<Q, Q::S.order[NS - 1]>(T, L, tp, it - 1) : cur;
      }
      bool active = true;
      if constexpr (maybe_inactive<kind>()) active = (live[s >> 5] >> (s & 31)) & 1u;
      if (active) {
        const float meff = cur.meff, bias = cur.bias;
        const float3 lin = cur.lin, angA = cur.angA, angB = cur.angB;
        const float la = cur.la, lb = cur.lb;
        const int br = cur.br;
        float ia[6], ib[6];
        if (a >= 0) {
#pragma unroll
          for (int q = 0; q < 6; ++q) ia[q] = S[T.sm_iinv + 6 * a + q];
        }
        if (b >= 0) {
#pragma unroll
          for (int q = 0; q < 6; ++q) ib[q] = S[T.sm_iinv + 6 * b + q];
        }
        const float dl = la - lb;
        float dbar = 0.f;
        float3 va = f3(0.f, 0.f, 0.f), wa = va, vb3 = va, wb3 = va, vba = va, wba = va, vbb = va, wbb = va;
        if (a >= 0) {
          const float3 IA = symv(ia, angA);
          const float c = dl * im[a];
          v[a][0] -= c * lin.x; v[a][1] -= c * lin.y; v[a][2] -= c * lin.z;
          v[a][3] -= dl * IA.x; v[a][4] -= dl * IA.y; v[a][5] -= dl * IA.z;
          va = f3(v[a][0], v[a][1], v[a][2]);
          wa = f3(v[a][3], v[a][4], v[a][5]);
          vba = VB.v3(6 * a);
          wba = VB.v3(6 * a + 3);
          dbar += im[a] * dot3(lin, vba) + dot3(IA, wba);
        }
        if (b >= 0) {
          const float3 IB = symv(ib, angB);
          const float c = dl * im[b];
          v[b][0] += c * lin.x; v[b][1] += c * lin.y; v[b][2] += c * lin.z;
          v[b][3] -= dl * IB.x; v[b][4] -= dl * IB.y; v[b][5] -= dl * IB.z;
          vb3 = f3(v[b][0], v[b][1], v[b][2]);
          wb3 = f3(v[b][3], v[b][4], v[b][5]);
          vbb = VB.v3(6 * b);
          wbb = VB.v3(6 * b + 3);
          dbar += -im[b] * dot3(lin, vbb) + dot3(IB, wbb);
        }
        float3 linb = dl * ((a >= 0 ? im[a] : 0.f) * vba - (b >= 0 ? im[b] : 0.f) * vbb);
        float3 angAb = f3(0.f, 0.f, 0.f), angBb = angAb;
        if (a >= 0) {
          const float3 g = dl * wba;
          angAb += symv(ia, g);
          float* q = ib9r[a];
          q[0] += g.x * angA.x; q[1] += g.x * angA.y; q[2] += g.x * angA.z;
          q[3] += g.y * angA.x; q[4] += g.y * angA.y; q[5] += g.y * angA.z;
          q[6] += g.z * angA.x; q[7] += g.z * angA.y; q[8] += g.z * angA.z;
          if constexpr (!lin_is_zero<kind>()) imbr[a] += dl * dot3(lin, vba);
        }
        if (b >= 0) {
          const float3 g = dl * wbb;
          angBb += symv(ib, g);
          float* q = ib9r[b];
          q[0] += g.x * angB.x; q[1] += g.x * angB.y; q[2] += g.x * angB.z;
          q[3] += g.y * angB.x; q[4] += g.y * angB.y; q[5] += g.y * angB.z;
          q[6] += g.z * angB.x; q[7] += g.z * angB.y; q[8] += g.z * angB.z;
          if constexpr (!lin_is_zero<kind>()) imbr[b] -= dl * dot3(lin, vbb);
        }
        const float lbar_a = S[T.sm_lam + s] + dbar;
        const int rc = s * RC_N;
        const float inside = br == 0 ? 1.f : 0.f;
        const float sg = br == 2 ? 1.f : (br == 1 ? -1.f : 0.f);
        const float pbar = inside * lbar_a;
        if constexpr (kind == RK_GT || kind == RK_PT) {
          constexpr int ns_ = Q::S.normal[s];
          RC[rc + RC_BND] += sg * cur.lnrm * lbar_a;
          S[T.sm_lam + ns_] += sg * cur.bnd * lbar_a;
        } else if constexpr (kind == RK_MOTOR) {
          RC[rc + RC_BND] += sg * lbar_a;
        }
        float Jv = 0.f;
        if (a >= 0) Jv += dot3(lin, va) + dot3(angA, wa);
        if (b >= 0) Jv += dot3(angB, wb3) - dot3(lin, vb3);
        RC[rc + RC_MEFF] += -pbar * (Jv + bias + gamma * lb);
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
          linb -= jvb * vb3;
          angBb += jvb * wb3;
        }
        if constexpr (!lin_is_constant<kind, Q::S.sub[s]>() && !lin_is_zero<kind>()) RC.a3(rc + RC_LIN, linb);
        if (a >= 0) RC.a3(rc + RC_ANGA, angAb);
        if (b >= 0) RC.a3(rc + RC_ANGB, angBb);
        S[T.sm_lam + s] = -dbar + pbar * (1.f - meff * gamma);
      }
      cur = nxt;
    });
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    S[T.sm_invmb + b] += imbr[b];
#pragma unroll
    for (int k = 0; k < 9; ++k) S[T.sm_iinvb + 9 * b + k] += ib9r[b][k];
  }
}
