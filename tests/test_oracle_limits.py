"""Pins of the oracle's joint-limit rows against mechanics (no GPU).

A uniform rod hangs from a world hinge about the y axis; its hinge angle is the rotation about
+y. Gravity's torque about the pivot is -(m g L / 2) sin(theta), and the hinge's reaction force
passes through the pivot, so the only other angular impulse about the pivot's axis is the
limit row's. That fixes, without the oracle's formulas:

* a rod released inside the range and falling onto its lower (upper) bound stops there: it goes
  past the bound by at most one step of its impact speed (the limit is detected at the start of
  a step; the speed follows from the energy of the fall) and comes to rest at the bound, up to
  the O(g h^2) step of the position correction;
* at rest the limit's mean impulse per step balances gravity's angular impulse,
  (m g L / 2) sin(bound) h;
* at an exact tie (angle equal to the bound, moving outward) the row is active and removes the
  rod's angular momentum about the pivot, I_p |omega| with I_p = I_yy + m (L / 2)^2;
* strictly inside the range the row is masked: the rollout equals that of the rod without a
  limit.

A flipped sign of the row's Jacobian or bias, or a wrong activation test, fails one of these.
"""
import math

import numpy as np

import oracle as O
from paper_1611_01652_gb300 import workloads as WL

G = 9.81
L_ROD, M_ROD, DT = 0.5, 1.0, 0.01


def rod(phi0, w0, lo, hi, limit=True, iters=100, horizon=300):
    m = WL.pendulum1(B=1, L=L_ROD, m=M_ROD, amp_deg=0.0, horizon=horizon, dt=DT, iters=iters)
    R = WL._rot_y(phi0)
    c = R @ np.array([0.0, 0.0, -L_ROD / 2])          # centre of mass relative to the pivot
    w = np.array([0.0, w0, 0.0])
    m.state0[0, 0] = WL.f32(WL._state(c, R, np.cross(w, c), w))
    m.joint_flags = np.array([1 if limit else 0], np.int32)
    m.limit[0, 0] = WL.f32([lo, hi])
    return m


def angle(x):
    """Rotation about +y of the rod's frame (its x axis against the world x axis)."""
    R = x[0, 3:12].reshape(3, 3)
    return math.atan2(-R[2, 0], R[0, 0])


def limit_slot(m):
    return int(np.flatnonzero(O.schedule(m)["kind"] == 2)[0])


def settle(m, steps):
    x = m.state0[0].astype(np.float64)
    s = limit_slot(m)
    th, lam, act = [], [], []
    for t in range(steps):
        x, a, _, l = O.step(m, 0, x, t=t)
        th.append(angle(x))
        lam.append(l[s])
        act.append(a[s])
    return np.array(th), np.array(lam), np.array(act), x


def impact_overshoot(phi0, bound):
    """One step of the angular speed reached by falling from phi0 to the bound (energy)."""
    dE = M_ROD * G * L_ROD / 2 * (math.cos(bound) - math.cos(phi0))
    return math.sqrt(2 * dE / pivot_inertia()) * DT


def pivot_inertia():
    return M_ROD * (3 * 0.005 ** 2 + L_ROD ** 2) / 12.0 + M_ROD * (L_ROD / 2) ** 2


def test_rod_falls_onto_lower_bound_and_rests_there():
    lo, hi = 0.2, 1.5
    th, lam, act, x = settle(rod(0.6, 0.0, lo, hi), 300)
    assert th.min() >= lo - 1.1 * impact_overshoot(0.6, lo), th.min()
    assert abs(th[-100:].mean() - lo) <= 2e-3, th[-100:].mean()
    assert act[-100:].any() and (lam >= 0.0).all()
    wy = x[0, 16]
    assert abs(wy) <= 0.05, wy                           # at rest (one limit-cycle step at most)
    tau = M_ROD * G * L_ROD / 2 * math.sin(lo) * DT      # gravity's angular impulse per step
    assert abs(lam[-100:].mean() - tau) <= 0.02 * tau, (lam[-100:].mean(), tau)


def test_rod_falls_onto_upper_bound_and_rests_there():
    lo, hi = -1.5, -0.2
    th, lam, act, x = settle(rod(-0.6, 0.0, lo, hi), 300)
    assert th.max() <= hi + 1.1 * impact_overshoot(-0.6, hi), th.max()
    assert abs(th[-100:].mean() - hi) <= 2e-3, th[-100:].mean()
    assert act[-100:].any() and (lam >= 0.0).all()
    tau = M_ROD * G * L_ROD / 2 * math.sin(-hi) * DT
    assert abs(lam[-100:].mean() - tau) <= 0.02 * tau, (lam[-100:].mean(), tau)


def test_tie_at_lower_bound_is_active_and_stops_the_rod():
    """Angle exactly at the bound (theta = 0: the rotation is the identity), moving outward."""
    m = rod(0.0, -1.0, 0.0, 1.0, iters=400)
    xn, a, _, lam = O.step(m, 0, m.state0[0], t=0)
    s = limit_slot(m)
    assert a[s] == 1
    Ip = pivot_inertia()
    assert abs(lam[s] - Ip * 1.0) <= 1e-3 * Ip, (lam[s], Ip)
    assert abs(xn[0, 16]) <= 1e-3                        # angular velocity about y removed


def test_tie_at_upper_bound_is_active_and_stops_the_rod():
    m = rod(0.0, 1.0, -1.0, 0.0, iters=400)
    xn, a, _, lam = O.step(m, 0, m.state0[0], t=0)
    s = limit_slot(m)
    assert a[s] == 1
    Ip = pivot_inertia()
    assert abs(lam[s] - Ip * 1.0) <= 1e-3 * Ip, (lam[s], Ip)
    assert abs(xn[0, 16]) <= 1e-3


def test_limit_inside_range_is_a_no_op():
    """A swing that stays inside (-0.5, 0.5) rad: the limited rod moves exactly as the free one."""
    lim, _, a, _ = O.rollout(rod(0.3, 0.0, -0.5, 0.5, iters=20, horizon=200), 0, log=True)
    free, _, _, _ = O.rollout(rod(0.3, 0.0, -0.5, 0.5, limit=False, iters=20, horizon=200), 0, log=True)
    m = rod(0.3, 0.0, -0.5, 0.5, iters=20, horizon=200)
    assert not a[:, limit_slot(m)].any()
    assert np.allclose(lim, free, rtol=0.0, atol=1e-12)
