// Reverse mode of the projected Gauss-Seidel sweeps split over the four warps of a CTA
// (compiled topologies, whole solver tape recorded by the rollout).
//
// The reverse of a sweep (section 2.1.1, back-propagation through the unrolled solver) has one
// sequential dependency: the adjoint of the velocities, carried from row to row in reverse sweep
// order, and the impulse adjoints carried from one sweep to the one before. Everything else a
// row contributes (the adjoints of its Jacobian, effective mass, bias and of the world inverse
// inertias) is a sum over sweeps that nothing in the sweep reads back. So:
//
//  * warp 0 (the chain) keeps the velocity adjoints of its 32 instances in registers (the
//    impulse adjoints in shared memory) and, per row, forms d = (M^-1 J^T) . v_bar, the clamped-branch
//    adjoint p_bar and j = -m_eff p_bar, updates v_bar += j J^T, and hands (j, p_bar) to the
//    others through a two-buffer ring in shared memory;
//  * warps 1..3 (the helpers) each own a fixed set of bodies (balanced at compile time by the
//    number of row sides touching them) and, one ring chunk behind the chain, replay the
//    velocities (undoing each row's impulse from the post-sweep values on the tape) and the
//    velocity adjoints of their bodies, and accumulate every row-side adjoint of those bodies;
//    the row-level adjoints (bias, the effective mass's bias and impulse terms) go with side a,
//    or with side b when the row's parent is the world.
//
// The four warps meet at one CTA barrier per chunk of DPK_MW_CH rows: in step k the chain
// writes chunk k into ring buffer k % 2 while the helpers read chunk k - 1 from the other
// buffer. Every warp executes the same number of barriers (one per chunk plus one), whatever
// its role, so the barrier sequence cannot deadlock.
#pragma once
#include "dp_static.cuh"

// CTA barrier 1 over the four warps (each warp arrives from its own code path).
__device__ __forceinline__ void mw_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Bodies owned by the three helper warps: longest-processing-time assignment by the number of
// row sides that touch each body (ties: lower body index, lower helper index).
struct MwOwn {
  int owner[DPK_MAXB];
  int load[3];
};
template <class Q>
constexpr MwOwn mw_owners() {
  MwOwn p{};
  int cnt[DPK_MAXB] = {};
  for (int s = 0; s < Q::NS; ++s) {
    if (Q::S.a[s] >= 0) ++cnt[Q::S.a[s]];
    if (Q::S.b[s] >= 0) ++cnt[Q::S.b[s]];
  }
  bool done[DPK_MAXB] = {};
  for (int k = 0; k < Q::NB; ++k) {
    int best = -1;
    for (int b = 0; b < Q::NB; ++b)
      if (!done[b] && (best < 0 || cnt[b] > cnt[best])) best = b;
    done[best] = true;
    int h = 0;
    for (int g = 1; g < 3; ++g)
      if (p.load[g] < p.load[h]) h = g;
    p.owner[best] = h;
    p.load[h] += cnt[best];
  }
  return p;
}
template <class Q>
struct MwPlan {
  static constexpr MwOwn own = mw_owners<Q>();
  static constexpr int NCH = (Q::NS + DPK_MW_CH - 1) / DPK_MW_CH;
  // rows whose linear Jacobian part is not a constant would need a row-level linear adjoint
  // split across two helpers; the compiled topologies have none (no sphere pairs)
  static constexpr bool lin_ok() {
    for (int s = 0; s < Q::NS; ++s)
      if (Q::S.kind[s] == RK_PN || Q::S.kind[s] == RK_PT) return false;
    return true;
  }
  static_assert(lin_ok(), "multi-warp reverse sweep: sphere-pair rows are not supported");
};

// Rows live on some lane of the warp (the same mask in every warp: same instances, same tape).
template <class Q>
__device__ __forceinline__ void mw_live(const LaneT<GSR>& L, unsigned (&live)[(Q::NS + 31) / 32]) {
  constexpr int NW = (Q::NS + 31) / 32;
#pragma unroll
  for (int w = 0; w < NW; ++w) live[w] = 0u;
  static_for<Q::NS>([&](auto SI) {
    constexpr int s = decltype(SI)::value;
    if constexpr (maybe_inactive<Q::S.kind[s]>()) {
      const float meff = L.rows.at(s * RF_N)[RF_MEFF];
      if (__any_sync(FULLMASK, meff != 0.f)) live[s >> 5] |= 1u << (s & 31);
    } else {
      live[s >> 5] |= 1u << (s & 31);
    }
  });
}

// Impulse of slot s before sweep `it` updated it.
template <class Q>
__device__ __forceinline__ float mw_lam_before(const DevTopo& T, const TapeStep& tp, int it, int s) {
  return it > 0 ? __ldg(tp.lam + ((it - 1) * Q::NS + s) * 32) : (T.ws ? __ldg(tp.lam0 + s * 32) : 0.f);
}

// Tape values the chain needs for one row.
struct MwChainIn {
  float meff, bnd, lnrm;
  float3 angA, angB, IA, IB;
  int br;
};
template <class Q, int s>
__device__ __forceinline__ MwChainIn mw_chain_load(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it) {
  constexpr int kind = Q::S.kind[s], a = Q::S.a[s], b = Q::S.b[s];
  const GSR R = L.rows.at(s * RF_N);
  MwChainIn r;
  r.meff = R[RF_MEFF];
  r.angA = a >= 0 ? R.v3(RF_ANGA) : f3(0.f, 0.f, 0.f);
  r.IA = a >= 0 ? R.v3(RF_IA) : f3(0.f, 0.f, 0.f);
  r.angB = b >= 0 ? R.v3(RF_ANGB) : f3(0.f, 0.f, 0.f);
  r.IB = b >= 0 ? R.v3(RF_IB) : f3(0.f, 0.f, 0.f);
  r.br = __ldg(tp.br + (it * Q::NS + s) * 32);
  r.bnd = 0.f;
  r.lnrm = 0.f;
  if constexpr (kind == RK_GT || kind == RK_PT) {
    // the normal impulse the friction row saw: after this sweep when the normal row comes
    // first in the sweep order, else before it
    constexpr int nrm = Q::S.normal[s];
    r.bnd = R[RF_BND];
    if constexpr (order_pos<Q>(nrm) < order_pos<Q>(s))
      r.lnrm = __ldg(tp.lam + (it * Q::NS + nrm) * 32);
    else
      r.lnrm = mw_lam_before<Q>(T, tp, it, nrm);
  }
  return r;
}

// Slot at reverse position ri (ri = 0 is the last row of a sweep).
template <class Q, int ri>
__device__ __forceinline__ constexpr int mw_slot() { return Q::S.order[Q::NS - 1 - ri]; }

// Depth of the tape look-ahead (rows of one warp's own sequence whose tape values are in flight
// while it works on the current one): enough to cover the L2 latency of the tape loads.
#define DPK_MW_AHEAD 8

// Tape values of chain position p (sweep it; positions beyond the sweep belong to sweep it - 1).
// The look-ahead register of position p is pre[p % DPK_MW_AHEAD]; it carries over into the next
// sweep only when the sweep's length is a multiple of the depth (the slots of the two sweeps'
// positions then line up); otherwise each sweep refills its first slots when it starts.
template <class Q, int p>
__device__ __forceinline__ void mw_chain_prefetch(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it,
                                                  MwChainIn& dst) {
  if constexpr (p < Q::NS) {
    dst = mw_chain_load<Q, mw_slot<Q, p>()>(T, L, tp, it);
  } else if constexpr (Q::NS % DPK_MW_AHEAD == 0 && p - Q::NS < Q::NS) {
    if (it > 0) dst = mw_chain_load<Q, mw_slot<Q, p - Q::NS>()>(T, L, tp, it - 1);
  }
}

// The chain warp: velocity and impulse adjoints through every sweep, last sweep first. On entry
// VB holds the adjoint of the solver's output velocities; on exit the adjoint of its input
// velocities. Also accumulates the bound adjoints (RC_BND) of friction and servo rows. The
// impulse adjoints live in the (otherwise unused) impulse array of shared memory.
template <class Q>
__device__ __noinline__ void pgs_reverse_chain(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp) {
  constexpr int NB = Q::NB, NS = Q::NS, CH = DPK_MW_CH, NCH = MwPlan<Q>::NCH, D = DPK_MW_AHEAD;
  constexpr int NW = (NS + 31) / 32;
  const SL S{g_smem + (threadIdx.x & 31)};
  const SL VB = S.at(T.sm_vb), RC = S.at(T.sm_rc), LB = S.at(T.sm_lam);
  float* ring0 = g_smem + (threadIdx.x & 31) + T.sm_ring * 32;
  const float gamma = T.gamma;
  const int iters = T.iters;
  unsigned live[NW];
  mw_live<Q>(L, live);
  float vb[NB][6], im[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    im[b] = S[T.sm_invm + b];
#pragma unroll
    for (int k = 0; k < 6; ++k) vb[b][k] = VB[6 * b + k];
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) LB[s] = 0.f;
  MwChainIn pre[D];
  static_for<D>([&](auto PI) { mw_chain_prefetch<Q, decltype(PI)::value>(T, L, tp, iters - 1, pre[decltype(PI)::value]); });
  for (int it = iters - 1; it >= 0; --it) {
    if constexpr (NS % D != 0) {
      if (it != iters - 1)
        static_for<D>([&](auto PI) { mw_chain_prefetch<Q, decltype(PI)::value>(T, L, tp, it, pre[decltype(PI)::value]); });
    }
    static_for<NCH>([&](auto QI) {
      constexpr int q = decltype(QI)::value;
      float* ring = ring0 + ((((iters - 1 - it) * NCH + q) & 1) * 2 * CH) * 32;
      static_for<CH>([&](auto JI) {
        constexpr int j = decltype(JI)::value;
        constexpr int ri = q * CH + j;
        if constexpr (ri < NS) {
          constexpr int s = mw_slot<Q, ri>();
          constexpr int kind = Q::S.kind[s], sub = Q::S.sub[s], a = Q::S.a[s], b = Q::S.b[s];
          const MwChainIn cur = pre[ri % D];
          mw_chain_prefetch<Q, ri + D>(T, L, tp, it, pre[ri % D]);
          bool active = true;
          if constexpr (maybe_inactive<kind>()) active = (live[s >> 5] >> (s & 31)) & 1u;
          if (active) {
            constexpr int ax = lin_axis<kind, sub>();  // a unit axis or none (no sphere pairs here)
            float dbar = 0.f;
            if constexpr (a >= 0) {
              const float wa = cur.IA.x * vb[a][3] + cur.IA.y * vb[a][4] + cur.IA.z * vb[a][5];
              if constexpr (ax >= 0) dbar += im[a] * vb[a][ax] + wa;
              else dbar += wa;
            }
            if constexpr (b >= 0) {
              const float wb = cur.IB.x * vb[b][3] + cur.IB.y * vb[b][4] + cur.IB.z * vb[b][5];
              if constexpr (ax >= 0) dbar += -im[b] * vb[b][ax] + wb;
              else dbar += wb;
            }
            const float lbar_a = LB[s] + dbar;  // adjoint of the row's new impulse
            const int br = cur.br;
            const float pbar = br == 0 ? lbar_a : 0.f;
            const float sg = br == 2 ? 1.f : (br == 1 ? -1.f : 0.f);
            if constexpr (kind == RK_GT || kind == RK_PT) {
              constexpr int nrm = Q::S.normal[s];
              RC[s * RC_N + RC_BND] += sg * cur.lnrm * lbar_a;
              LB[nrm] += sg * cur.bnd * lbar_a;
            } else if constexpr (kind == RK_MOTOR) {
              RC[s * RC_N + RC_BND] += sg * lbar_a;
            }
            const float meff = cur.meff;
            const float jvb = -meff * pbar;
            if constexpr (a >= 0) {
              if constexpr (ax >= 0) vb[a][ax] += jvb;
              vb[a][3] = fmaf(jvb, cur.angA.x, vb[a][3]); vb[a][4] = fmaf(jvb, cur.angA.y, vb[a][4]);
              vb[a][5] = fmaf(jvb, cur.angA.z, vb[a][5]);
            }
            if constexpr (b >= 0) {
              if constexpr (ax >= 0) vb[b][ax] -= jvb;
              vb[b][3] = fmaf(jvb, cur.angB.x, vb[b][3]); vb[b][4] = fmaf(jvb, cur.angB.y, vb[b][4]);
              vb[b][5] = fmaf(jvb, cur.angB.z, vb[b][5]);
            }
            LB[s] = -dbar + pbar * (1.f - meff * gamma);
            ring[j * 32] = jvb;
            ring[(CH + j) * 32] = pbar;
          }
        }
      });
      mw_barrier();
    });
  }
  mw_barrier();  // the helpers' last chunk
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int k = 0; k < 6; ++k) VB[6 * b + k] = vb[b][k];
}

// Tape values a helper needs for one side of a row.
struct MwSideIn {
  float la, lb, bias;
  float3 ang, I;
};
// Number of bodies owned by helper H, and the k-th of them.
template <class Q, int H>
__device__ __forceinline__ constexpr int mw_nown() {
  int n = 0;
  for (int b = 0; b < Q::NB; ++b) n += MwPlan<Q>::own.owner[b] == H;
  return n;
}
template <class Q, int H>
__device__ __forceinline__ constexpr int mw_local(int body) {
  int n = 0;
  for (int b = 0; b < body; ++b) n += MwPlan<Q>::own.owner[b] == H;
  return n;
}

// The row sides of helper H's bodies in reverse sweep order: reverse position and side. The
// helper's loop is unrolled over this sequence, so slots, sides and its bodies' registers are
// compile-time constants, and the tape values of the next DPK_MW_AHEAD row sides are in flight
// while it works on the current one (continuing across chunk and sweep boundaries).
struct MwSeq {
  int n;
  int ri[2 * DPK_MAXSLOT];
  bool side_a[2 * DPK_MAXSLOT];
};
template <class Q, int H>
constexpr MwSeq mw_seq() {
  MwSeq q{};
  for (int ri = 0; ri < Q::NS; ++ri) {
    const int s = Q::S.order[Q::NS - 1 - ri];
    if (Q::S.a[s] >= 0 && MwPlan<Q>::own.owner[Q::S.a[s]] == H) { q.ri[q.n] = ri; q.side_a[q.n] = true; ++q.n; }
    if (Q::S.b[s] >= 0 && MwPlan<Q>::own.owner[Q::S.b[s]] == H) { q.ri[q.n] = ri; q.side_a[q.n] = false; ++q.n; }
  }
  return q;
}
template <class Q, int H>
struct MwSeqOf {
  static constexpr MwSeq seq = mw_seq<Q, H>();
  // first sequence position of chunk c (c = NCH: the end)
  __host__ __device__ static constexpr int first(int c) {
    int k = 0;
    while (k < seq.n && seq.ri[k] < c * DPK_MW_CH) ++k;
    return k;
  }
};

// Tape values a helper needs for one side of a row.
template <class Q, int s, bool SIDE_A>
__device__ __forceinline__ MwSideIn mw_side_load(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it) {
  const GSR R = L.rows.at(s * RF_N);
  MwSideIn r;
  r.la = __ldg(tp.lam + (it * Q::NS + s) * 32);
  r.lb = mw_lam_before<Q>(T, tp, it, s);
  r.bias = (SIDE_A || Q::S.a[s] < 0) ? R[RF_BIAS] : 0.f;  // the side carrying the row-level terms
  r.ang = R.v3(SIDE_A ? RF_ANGA : RF_ANGB);
  r.I = R.v3(SIDE_A ? RF_IA : RF_IB);
  return r;
}

// Tape values of helper sequence position p (sweep it; beyond the sequence: sweep it - 1), with
// the chain's rule for carrying the look-ahead into the next sweep.
template <class Q, int H, int p>
__device__ __forceinline__ void mw_side_prefetch(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it,
                                                 MwSideIn& dst) {
  constexpr MwSeq sq = MwSeqOf<Q, H>::seq;
  if constexpr (p < sq.n) {
    dst = mw_side_load<Q, mw_slot<Q, sq.ri[p]>(), sq.side_a[p]>(T, L, tp, it);
  } else if constexpr (sq.n % DPK_MW_AHEAD == 0 && p - sq.n < sq.n) {
    if (it > 0) dst = mw_side_load<Q, mw_slot<Q, sq.ri[p - sq.n]>(), sq.side_a[p - sq.n]>(T, L, tp, it - 1);
  }
}

// One row side (body x = a or b of slot s, owned by this helper): velocities before the row's
// impulse (undoing v += M^-1 J^T dl from the post-sweep values), the side's Jacobian,
// effective-mass, bias and inverse-inertia adjoints, then the velocity adjoint after the chain's
// update of the row (the same arithmetic as the chain).
template <class Q, int s, bool SIDE_A>
__device__ __forceinline__ void mw_side(const DevTopo& T, const SL& RC, const MwSideIn& in, float jvb, float pbar,
                                        float (&v)[6], float (&vb)[6], const float (&ii)[6], float im,
                                        float (&ib9)[9], float& imb) {
  constexpr int kind = Q::S.kind[s], sub = Q::S.sub[s];
  constexpr int ax = lin_axis<kind, sub>();  // the linear part: a unit axis or none
  const float sgn = SIDE_A ? 1.f : -1.f;  // J_v = +lin on side a, -lin on side b
  const float dl = in.la - in.lb;
  const float c = dl * im;
  if constexpr (ax >= 0) v[ax] -= sgn * c;
  v[3] -= dl * in.I.x; v[4] -= dl * in.I.y; v[5] -= dl * in.I.z;
  // adjoint of M^-1 J^T: dl * v_bar (before the chain's update of this row)
  const float3 g = f3(dl * vb[3], dl * vb[4], dl * vb[5]);
  float3 angb = symv(ii, g);
  ib9[0] += g.x * in.ang.x; ib9[1] += g.x * in.ang.y; ib9[2] += g.x * in.ang.z;
  ib9[3] += g.y * in.ang.x; ib9[4] += g.y * in.ang.y; ib9[5] += g.y * in.ang.z;
  ib9[6] += g.z * in.ang.x; ib9[7] += g.z * in.ang.y; ib9[8] += g.z * in.ang.z;
  if constexpr (ax >= 0) imb += sgn * dl * vb[ax];
  // Jacobian adjoint from the row's J v term, and this side's share of J v
  angb += jvb * f3(v[3], v[4], v[5]);
  const float wj = in.ang.x * v[3] + in.ang.y * v[4] + in.ang.z * v[5];
  float jv = wj;
  if constexpr (ax >= 0) jv = sgn * v[ax] + wj;
  const int rc = s * RC_N;
  if constexpr (SIDE_A) {
    RC.a3(rc + RC_ANGA, angb);
    RC[rc + RC_MEFF] += -pbar * (jv + in.bias + T.gamma * in.lb);
    RC[rc + RC_BIAS] += jvb;
  } else if constexpr (Q::S.a[s] < 0) {
    // the row's parent is the world: side b carries the row-level terms
    RC.a3(rc + RC_ANGB, angb);
    RC[rc + RC_MEFF] += -pbar * (jv + in.bias + T.gamma * in.lb);
    RC[rc + RC_BIAS] += jvb;
  } else {
    RC.a3(rc + RC_ANGB, angb);
    RC[rc + RC_LIN] += -pbar * jv;  // side b's share of the effective-mass adjoint (folded later)
  }
  if constexpr (ax >= 0) vb[ax] += sgn * jvb;
  vb[3] = fmaf(jvb, in.ang.x, vb[3]); vb[4] = fmaf(jvb, in.ang.y, vb[4]); vb[5] = fmaf(jvb, in.ang.z, vb[5]);
}

// Helper H: one chunk (sweep it, chunk q) of the rows, for the sides of its bodies.
template <class Q, int H, int q, int NO>
__device__ __forceinline__ void mw_helper_chunk(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int it,
                                                const float* ring, const unsigned* live, const SL& RC,
                                                MwSideIn (&pre)[DPK_MW_AHEAD], float (&v)[NO][6], float (&vb)[NO][6],
                                                const float (&ii)[NO][6], const float (&im)[NO], float (&ib9)[NO][9],
                                                float (&imb)[NO]) {
  constexpr int CH = DPK_MW_CH, D = DPK_MW_AHEAD;
  constexpr MwSeq sq = MwSeqOf<Q, H>::seq;
  constexpr int p0 = MwSeqOf<Q, H>::first(q), p1 = MwSeqOf<Q, H>::first(q + 1);
  if constexpr (q == 0) {
    // a sweep whose length is not a multiple of the look-ahead depth refills its first slots
    if constexpr (sq.n % D != 0) {
      if (it != T.iters - 1)
        static_for<D>([&](auto PI) { mw_side_prefetch<Q, H, decltype(PI)::value>(T, L, tp, it, pre[decltype(PI)::value]); });
    }
    // the velocities after sweep it (the reverse sweep undoes its rows from there)
    const float* vi = tp.viter + it * Q::NB * 6 * 32;
    static_for<Q::NB>([&](auto BI) {
      constexpr int bd = decltype(BI)::value;
      if constexpr (MwPlan<Q>::own.owner[bd] == H) {
        constexpr int k = mw_local<Q, H>(bd);
#pragma unroll
        for (int f = 0; f < 6; ++f) v[k][f] = __ldg(vi + (6 * bd + f) * 32);
      }
    });
  }
  static_for<p1 - p0>([&](auto PI) {
    constexpr int p = p0 + decltype(PI)::value;
    constexpr int ri = sq.ri[p];
    constexpr bool sideA = sq.side_a[p];
    constexpr int s = mw_slot<Q, ri>();
    constexpr int kind = Q::S.kind[s];
    constexpr int x = sideA ? Q::S.a[s] : Q::S.b[s];
    constexpr int k = mw_local<Q, H>(x);
    constexpr int j = ri - q * CH;
    const MwSideIn in = pre[p % D];
    mw_side_prefetch<Q, H, p + D>(T, L, tp, it, pre[p % D]);
    bool active = true;
    if constexpr (maybe_inactive<kind>()) active = (live[s >> 5] >> (s & 31)) & 1u;
    if (active) {
      const float jvb = ring[j * 32], pbar = ring[(CH + j) * 32];
      mw_side<Q, s, sideA>(T, RC, in, jvb, pbar, v[k], vb[k], ii[k], im[k], ib9[k], imb[k]);
    }
  });
}

// Helper warp H over every sweep, one ring chunk behind the chain. On exit its bodies'
// inverse-inertia and inverse-mass adjoints have been added to IINVB / INVMB.
template <class Q, int H>
__device__ __noinline__ void pgs_reverse_helper(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp) {
  constexpr int NB = Q::NB, NS = Q::NS, CH = DPK_MW_CH, NCH = MwPlan<Q>::NCH, D = DPK_MW_AHEAD;
  constexpr int NW = (NS + 31) / 32;
  constexpr int NO = mw_nown<Q, H>() > 0 ? mw_nown<Q, H>() : 1;
  const SL S{g_smem + (threadIdx.x & 31)};
  const SL VB = S.at(T.sm_vb), RC = S.at(T.sm_rc);
  const float* ring0 = g_smem + (threadIdx.x & 31) + T.sm_ring * 32;
  const int iters = T.iters;
  unsigned live[NW];
  mw_live<Q>(L, live);
  float v[NO][6], vb[NO][6], ii[NO][6], im[NO], ib9[NO][9], imb[NO];
  static_for<NB>([&](auto BI) {
    constexpr int bd = decltype(BI)::value;
    if constexpr (MwPlan<Q>::own.owner[bd] == H) {
      constexpr int k = mw_local<Q, H>(bd);
      im[k] = S[T.sm_invm + bd];
      imb[k] = 0.f;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        vb[k][f] = VB[6 * bd + f];
        ii[k][f] = S[T.sm_iinv + 6 * bd + f];
        v[k][f] = 0.f;
      }
#pragma unroll
      for (int f = 0; f < 9; ++f) ib9[k][f] = 0.f;
    }
  });
  MwSideIn pre[D];
  static_for<D>([&](auto PI) { mw_side_prefetch<Q, H, decltype(PI)::value>(T, L, tp, iters - 1, pre[decltype(PI)::value]); });
  for (int it = iters - 1; it >= 0; --it) {
    static_for<NCH>([&](auto QI) {
      constexpr int q = decltype(QI)::value;
      // the chunk the chain finished in the previous barrier interval
      if constexpr (q > 0) {
        const float* ring = ring0 + ((((iters - 1 - it) * NCH + q - 1) & 1) * 2 * CH) * 32;
        mw_helper_chunk<Q, H, q - 1>(T, L, tp, it, ring, live, RC, pre, v, vb, ii, im, ib9, imb);
      } else if (it + 1 < iters) {
        const float* ring = ring0 + ((((iters - 2 - it) * NCH + NCH - 1) & 1) * 2 * CH) * 32;
        mw_helper_chunk<Q, H, NCH - 1>(T, L, tp, it + 1, ring, live, RC, pre, v, vb, ii, im, ib9, imb);
      }
      mw_barrier();
    });
  }
  {
    const float* ring = ring0 + ((((iters - 1) * NCH + NCH - 1) & 1) * 2 * CH) * 32;
    mw_helper_chunk<Q, H, NCH - 1>(T, L, tp, 0, ring, live, RC, pre, v, vb, ii, im, ib9, imb);
  }
  mw_barrier();
  static_for<NB>([&](auto BI) {
    constexpr int bd = decltype(BI)::value;
    if constexpr (MwPlan<Q>::own.owner[bd] == H) {
      constexpr int k = mw_local<Q, H>(bd);
      S[T.sm_invmb + bd] += imb[k];
#pragma unroll
      for (int f = 0; f < 9; ++f) S[T.sm_iinvb + 9 * bd + f] += ib9[k][f];
    }
  });
}

// The whole reverse sweep on the CTA's four warps. Called by every warp; ends after a CTA
// barrier with VB, RC, IINVB and INVMB complete (RC_LIN's x field folded into RC_MEFF).
template <class Q>
__device__ void pgs_reverse_mw(const DevTopo& T, const LaneT<GSR>& L, const TapeStep& tp, int warp) {
  if (warp == 0)
    pgs_reverse_chain<Q>(T, L, tp);
  else if (warp == 1)
    pgs_reverse_helper<Q, 0>(T, L, tp);
  else if (warp == 2)
    pgs_reverse_helper<Q, 1>(T, L, tp);
  else
    pgs_reverse_helper<Q, 2>(T, L, tp);
  mw_barrier();
  // fold side b's effective-mass share (slots split over the warps; each slot by one warp)
  const SL RC{g_smem + (threadIdx.x & 31) + T.sm_rc * 32};
  for (int s = warp; s < Q::NS; s += 4) {
    RC[s * RC_N + RC_MEFF] += RC[s * RC_N + RC_LIN];
    RC[s * RC_N + RC_LIN] = 0.f;
  }
  mw_barrier();
}

// ------------------------------------------------------------------------------------------
// Stages after the sweeps, split over the four warps by body ownership (DevTopo.mw_own): warp w
// adds the row-side adjoints of the bodies it owns, and the joint-level adjoints (hinge axis,
// angle and servo-target adjoints, joint parameters) of the joints whose child body it owns;
// contact parameters go with the sphere's body. Every accumulator has one writer, and each
// writer takes the slots in slot order, so the sums are deterministic. Same arithmetic as
// ws_apply_reverse and rows_reverse; rows with a non-constant linear Jacobian part (sphere
// pairs) are not handled here (the multi-warp kernel is built only for topologies without them).

// The row record of slot s (18 lines) into L1.
__device__ __forceinline__ void mw_row_prefetch(const float* rows, int s) {
#pragma unroll
  for (int f = 0; f < RF_N; ++f) prefetch_l1(rows + (s * RF_N + f) * 32);
}
// The Jacobian lines of slot s (linear and both angular parts) into L1.
__device__ __forceinline__ void mw_jac_prefetch(const float* rows, int s) {
#pragma unroll
  for (int f = RF_LIN; f < RF_IA; ++f) prefetch_l1(rows + (s * RF_N + f) * 32);
}
// The per-instance parameter lines the row-assembly reverse of slot s reads, into L1 (the
// parameter array stays in L2 across steps; each field of a group is one 128-byte line).
__device__ __forceinline__ void mw_param_prefetch(const DevTopo& T, const float* prm, int s) {
  const int idx = T.sidx[s], Bp = T.Bp;
  int f0 = -1, nf = 0;
  switch (T.skind[s]) {
    case RK_JLIN: f0 = T.o_anchor + 6 * idx; nf = 6; break;
    case RK_JANG: f0 = T.o_axis + 6 * idx; nf = 6; break;
    case RK_LIMIT: f0 = T.o_limit + 2 * idx; nf = 1; break;
    case RK_GN:
    case RK_GT:
      f0 = T.o_sph_off + 3 * idx; nf = 3;
      prefetch_l1(prm + (size_t)(T.o_sph_rad + idx) * Bp);
      if (T.skind[s] == RK_GN) prefetch_l1(prm + (size_t)(T.o_sph_e + idx) * Bp);
      break;
    default: break;
  }
  for (int f = 0; f < nf; ++f) prefetch_l1(prm + (size_t)(f0 + f) * Bp);
}

// Reverse of the warm-start application v += M^-1 J^T lambda0, the sides this warp owns.
template <class RV>
__device__ void ws_apply_reverse_own(const DevTopo& T, const LaneT<RV>& L, const SL& VB, const SL& RC,
                                     const TapeStep& tp, int w) {
  const SL& S = L.S;
  // the starting impulses of every slot this warp owns a side of, then the Jacobian lines of
  // the slots two places ahead in the warp's list, into L1 ahead of their loads
  const int n = T.mw_nslot[w];
  const int16_t* lst = T.mw_slot[w];
  for (int k = 0; k < n; ++k) prefetch_l1(tp.lam0 + (lst[k] & 0xfff) * 32);
  for (int k = 0; k < 2 && k < n; ++k) mw_jac_prefetch(L.rows.p, lst[k] & 0xfff);
  for (int k = 0; k < n; ++k) {
    if (k + 2 < n) mw_jac_prefetch(L.rows.p, lst[k + 2] & 0xfff);
    const int e = lst[k], s = e & 0xfff;
    const int a = T.sa[s], b = T.sb[s];
    const bool oa = e & MW_SLOT_A, ob = e & MW_SLOT_B;
    const float dl = tp.lam0[s * 32];
    if (dl == 0.f) continue;
    const RV R = L.rows.at(s * RF_N);
    const int rc = s * RC_N;
    const float3 lin = R.v3(RF_LIN);
    if (oa) {
      const float3 vba = VB.v3(6 * a), g = dl * VB.v3(6 * a + 3), angA = R.v3(RF_ANGA);
      float ia[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ia[q] = S[T.sm_iinv + 6 * a + q];
      RC.a3(rc + RC_ANGA, symv(ia, g));
      add_outer(S, T.sm_iinvb + 9 * a, g, angA);
      S[T.sm_invmb + a] += dl * dot3(lin, vba);
    }
    if (ob) {
      const float3 vbb = VB.v3(6 * b), g = dl * VB.v3(6 * b + 3), angB = R.v3(RF_ANGB);
      float ib[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ib[q] = S[T.sm_iinv + 6 * b + q];
      RC.a3(rc + RC_ANGB, symv(ib, g));
      add_outer(S, T.sm_iinvb + 9 * b, g, angB);
      S[T.sm_invmb + b] -= dl * dot3(lin, vbb);
    }
  }
}

// Row adjoints pushed back to positions, rotations, the solver's input velocities
// (restitution), hinge axes/angles, servo targets and parameters: the parts this warp owns.

template <class RV>
__device__ void rows_reverse_own(const DevTopo& T, const BLaneT<RV>& B, const SL& XB, const SL& VB, const SL& RC, int w) {
  const LaneT<RV>& L = B.L;
  const SL& S = L.S;
  const float h = T.dt;
  const float bh = T.beta / h;
  const float3 ez = f3(0.f, 0.f, 1.f);
  // the row and parameter lines of the slots two places ahead in the warp's list into L1
  const int n = T.mw_nslot[w];
  const int16_t* lst = T.mw_slot[w];
  for (int k = 0; k < 2 && k < n; ++k) {
    mw_row_prefetch(L.rows.p, lst[k] & 0xfff);
    mw_param_prefetch(T, L.P.p, lst[k] & 0xfff);
  }
  for (int k = 0; k < n; ++k) {
    if (k + 2 < n) {
      mw_row_prefetch(L.rows.p, lst[k + 2] & 0xfff);
      mw_param_prefetch(T, L.P.p, lst[k + 2] & 0xfff);
    }
    const int e = lst[k], s = e & 0xfff;
    const int kind = T.skind[s], idx = T.sidx[s], sub = T.ssub[s], a = T.sa[s], b = T.sb[s];
    const bool oa = e & MW_SLOT_A, ob = e & MW_SLOT_B;
    const RV R = L.rows.at(s * RF_N);
    const float meff = R[RF_MEFF];
    if (meff == 0.f) continue;  // inactive on this lane: constant row
    const int rc = s * RC_N;
    const float3 lin = R.v3(RF_LIN);
    const float3 angA = R.v3(RF_ANGA), angB = R.v3(RF_ANGB);
    float3 angAb = RC.v3(rc + RC_ANGA), angBb = RC.v3(rc + RC_ANGB);
    const float biasb = RC[rc + RC_BIAS];
    // effective mass 1/(K + gamma)
    const float Kb = -meff * meff * RC[rc + RC_MEFF];
    if (a >= 0) {
      angAb += (2.f * Kb) * R.v3(RF_IA);
      if (oa) {
        add_outer(S, T.sm_iinvb + 9 * a, Kb * angA, angA);
        S[T.sm_invmb + a] += Kb * dot3(lin, lin);
      }
    }
    if (b >= 0) {
      angBb += (2.f * Kb) * R.v3(RF_IB);
      if (ob) {
        add_outer(S, T.sm_iinvb + 9 * b, Kb * angB, angB);
        S[T.sm_invmb + b] += Kb * dot3(lin, lin);
      }
    }
    switch (kind) {
      case RK_JLIN: {
        const float3 e = f3(sub == 0 ? 1.f : 0.f, sub == 1 ? 1.f : 0.f, sub == 2 ? 1.f : 0.f);
        const float3 Cb = (bh * biasb) * e;
        if (oa) {
          const float3 rab = cross3(e, angAb) + Cb;
          const M3 Ra = loadRg(B.X0, 18 * a);
          XB.a3(18 * a, Cb);
          add_outer(XB, 18 * a + 3, rab, L.P.v3(T.o_anchor + 6 * idx));
          B.G.red3(T.o_anchor + 6 * idx, mtv(Ra, rab));
        } else if (a < 0 && ob) {  // world anchor: its gradient goes with the child body
          B.G.red3(T.o_anchor + 6 * idx, cross3(e, angAb) + Cb);
        }
        if (ob) {
          const float3 rbb = -cross3(e, angBb) - Cb;
          const M3 Rb = loadRg(B.X0, 18 * b);
          XB.a3(18 * b, -Cb);
          add_outer(XB, 18 * b + 3, rbb, L.P.v3(T.o_anchor + 6 * idx + 3));
          B.G.red3(T.o_anchor + 6 * idx + 3, mtv(Rb, rbb));
        }
        break;
      }
      case RK_JANG: {
        float3 t1, t2;
        onb3(L.P.v3(T.o_axis + 6 * idx), t1, t2);
        const float3 tau = sub == 0 ? t1 : t2;
        const M3 Ra = body_Rg(B.X0, a), Rb = loadRg(B.X0, 18 * b);
        const float3 t = mv(Ra, tau);
        const float3 axb = L.P.v3(T.o_axis + 6 * idx + 3);
        const float3 ub = mv(Rb, axb);
        const float3 ua = S.v3(T.sm_ua + 3 * idx);
        if (oa) {
          const float3 cr = cross3(ub, ua);
          addR_outer(XB, a, angAb - angBb + (bh * biasb) * cr, tau);
        }
        if (ob) {
          const float3 crb = (bh * biasb) * t;
          S.a3(T.sm_uab + 3 * idx, cross3(crb, ub));      // c = ub x ua
          add_outer(XB, 18 * b + 3, cross3(ua, crb), axb);
        }
        break;
      }
      case RK_LIMIT: {
        if (!ob) break;
        const float th = S[T.sm_th + idx];
        const float lo_j = L.P[T.o_limit + 2 * idx];
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
        if (!ob) break;
        S.a3(T.sm_uab + 3 * idx, angBb - (a >= 0 ? angAb : f3(0.f, 0.f, 0.f)));
        S[T.sm_wstb + idx] -= biasb;
        B.G.red(T.o_motor + 3 * idx + 1, h * RC[rc + RC_BND]);
        break;
      }
      case RK_GN:
      case RK_GT: {
        const M3 Ra = loadRg(B.X0, 18 * a);
        const float3 off = L.P.v3(T.o_sph_off + 3 * idx);
        const float3 c = mv(Ra, off);
        const float rad = L.P[T.o_sph_rad + idx];
        const float d = (B.X0[18 * a + 2] + c.z) - rad - T.ground_z;
        float db = 0.f;
        if (kind == RK_GN) {
          const float3 vm = B.vminus.v3(6 * a), wm = B.vminus.v3(6 * a + 3);
          const float vn = dot3(lin, vm) + dot3(angA, wm);
          if (d + T.slop < 0.f) db += bh * biasb;
          if (vn < 0.f) {
            const float e = L.P[T.o_sph_e + idx];
            B.G.red(T.o_sph_e + idx, vn * biasb);
            const float vnb = e * biasb;
            VB.a3(6 * a, vnb * lin);
            VB.a3(6 * a + 3, vnb * angA);
            angAb += vnb * wm;
          }
        } else {
          B.G.red(T.o_sph_mu + idx, RC[rc + RC_BND]);
        }
        const float3 rab = cross3(lin, angAb);  // angA = ra x lin (lin constant)
        const float3 cb = rab + f3(0.f, 0.f, db);
        XB[18 * a + 2] += db;
        add_outer(XB, 18 * a + 3, cb, off);
        B.G.red3(T.o_sph_off + 3 * idx, mtv(Ra, cb));
        B.G.red(T.o_sph_rad + idx, -rab.z - db);
        break;
      }
      default:
        break;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Forward stages split over the four warps (the four-warp rollout kernel).

// The damped previous-impulse start (zero network, no harvest): warp w takes the row groups
// g = w, w + 4, ... (their starting impulses, projected) and the limit slots s = w, w + 4, ...
// (which start cold); after a CTA barrier it adds v += M^-1 J^T lambda0 to the bodies it owns
// (bmask), slot by slot in slot order, and records slots s = w, w + 4, ... of lambda0 on the
// tape. The same values as warm_start, in the same order per body.
template <bool TAPE, class RV>
__device__ void warm_start_mw(const DevTopo& T, const LaneT<RV>& L, const SL& X, const TapeStep& tp, int w,
                              uint32_t bmask) {
  const SL& S = L.S;
  for (int g = w; g < T.n_wsg; g += 4) {
    float z[3];
    for (int k = 0; k < 3; ++k) {
      const int s = T.wsg_slot[g][k];
      z[k] = T.ws_alpha * (s >= 0 ? S[T.sm_lam + s] : 0.f);
    }
    ws_project(T, L, g, z);
  }
  for (int s = w; s < T.nslots; s += 4)
    if (T.skind[s] == RK_LIMIT) S[T.sm_lam + s] = 0.f;
  mw_barrier();
  for (int s = 0; s < T.nslots; ++s) {
    const float l0 = S[T.sm_lam + s];
    if (l0 != 0.f) row_apply(T, S, L.rows.at(s * RF_N), X, T.sa[s], T.sb[s], l0, bmask);
  }
  if (TAPE)
    for (int s = w; s < T.nslots; s += 4) tp.lam0[s * 32] = S[T.sm_lam + s];
}
