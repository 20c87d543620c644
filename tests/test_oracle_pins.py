"""Pins of the FP64 oracle against facts fixed by the paper or by mechanics (no GPU).

Each test names what it pins. None re-types an oracle formula: the expected values are
closed forms of the discrete dynamics, conservation laws, printed numbers, library routines
(torch's bfloat16 conversion) or finite differences of the oracle's own forward pass.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1611_01652_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")
G = 9.81


# ----------------------------------------------------------------------------- bookkeeping
def test_param_counts_match_paper():
    """Controller sizes printed in sections 3.2.1, 3.2.2 and 3.3."""
    gold = json.load(open(GOLDEN))
    for e in gold["mlp_param_counts"]:
        assert O.param_count(e["widths"], e["skip"]) == e["count"], e["cite"]
        assert WL.param_count(e["widths"], e["skip"]) == e["count"], e["cite"]
    # the controllers of the benchmark workloads
    assert O.param_count([24, 128, 128, 8]) == 20744
    assert O.param_count([32, 256, 256, 7]) == 76039
    assert O.param_count([64, 1024, 1024, 8]) == 1124360


def test_table1_arithmetic():
    """Table 1: ms per robot-step = seconds / (robots x 1000 steps)."""
    gold = json.load(open(GOLDEN))
    steps = gold["table1_steps_per_simulation"]["steps"]
    assert steps == round(gold["table1_steps_per_simulation"]["seconds_simulated"] / gold["table1_steps_per_simulation"]["dt"])
    for e in gold["table1_ms_per_robot_step"]:
        assert abs(e["seconds"] * 1e3 / (e["robots"] * steps) - e["ms"]) <= 0.006, e["cite"]


def test_bf16_rounding_matches_torch():
    """The oracle's bfloat16 rounding equals torch's float32 -> bfloat16 conversion (RNE)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        # exact ties between two bfloat16 values
                        (np.arange(-300, 300) + 0.5) * 2.0 ** -7 + 1.0]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.bf16(float(v)) for v in x])
    assert np.array_equal(ref, got)


# ----------------------------------------------------------------------------- schedule
def test_schedule_is_a_valid_colouring():
    """Rows sharing a non-world body get different colours; sweep = (colour, slot) order;
    the quadruped has 80 slots (8x5 joint rows, 8 limits, 8 motors, 8 spheres x 3)."""
    m = WL.quadruped(B=1)
    s = O.schedule(m)
    n = len(s["kind"])
    assert n == 80
    for i in range(n):
        for k in range(i):
            bi = {s["body_a"][i], s["body_b"][i]} - {-1}
            bk = {s["body_a"][k], s["body_b"][k]} - {-1}
            if bi & bk:
                assert s["colour"][i] != s["colour"][k]
    key = [(s["colour"][j], j) for j in s["order"]]
    assert key == sorted(key)
    # the torso takes part in 40 rows, so at least 40 colours; greedy reaches that bound
    assert s["colour"].max() + 1 == 40


# ----------------------------------------------------------------------------- closed forms
def _high_ball(v0, w0=(0, 0, 0), z0=50.0, horizon=100):
    m = WL.ball(B=1, horizon=horizon)
    m.state0[0, 0, 2] = z0
    m.state0[0, 0, 12:15] = v0
    m.state0[0, 0, 15:18] = w0
    return m


def test_flight_is_discrete_symplectic_euler():
    """Free flight: v_z(n) = v_z0 - n g h, z(n) = z0 + n h v_z0 - g h^2 n(n+1)/2, x, y linear."""
    v0 = np.array([1.5, -2.0, 3.0])
    m = _high_ball(v0)
    st, _, act, _ = O.rollout(m, 0, log=True)
    assert act.sum() == 0
    h = m.dt
    n = np.arange(st.shape[0])
    z = 50.0 + n * h * v0[2] - G * h * h * n * (n + 1) / 2
    np.testing.assert_allclose(st[:, 0, 2], z, rtol=1e-12)
    np.testing.assert_allclose(st[:, 0, 14], v0[2] - n * G * h, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st[:, 0, 0], n * h * v0[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st[:, 0, 1], n * h * v0[1], rtol=1e-12, atol=1e-12)


def test_flight_gradient_closed_form():
    """Before any contact, p_T = p_0 + T h v_0 + const, so d|p_T - y|^2 / dv_0 = 2 (p_T - y) T h."""
    m = _high_ball(np.array([1.0, 2.0, 0.5]), horizon=40)
    L, g = O.rollout_grad(m, 0)
    st, _, _, _ = O.rollout(m, 0)
    expect = 2.0 * (st[-1, 0, :3] - m.loss_target[0]) * 40 * m.dt
    np.testing.assert_allclose(g["state0"][0, 12:15], expect, rtol=1e-12)
    np.testing.assert_allclose(g["state0"][0, 0:3], 2.0 * (st[-1, 0, :3] - m.loss_target[0]), rtol=1e-12)


def test_sliding_friction_closed_form():
    """A sphere sliding on the ground at rest height r - slop (zero Baumgarte bias): the normal
    impulse is m g h, the friction impulse mu m g h, so v_x(n) = v0 - n mu g h and
    w_y(n) = n mu m g h r / I (= n 5 mu g h / (2 r)) until the contact point stops slipping."""
    m = WL.ball(B=1, horizon=15)
    r, mu, h = float(m.sph_rad[0, 0]), float(m.sph_mu[0, 0]), m.dt
    m.state0[0, 0, 2] = r - m.slop
    m.state0[0, 0, 12:15] = [3.0, 0.0, 0.0]
    m.state0[0, 0, 15:18] = 0.0
    st, _, act, _ = O.rollout(m, 0, log=True)
    assert act.all()
    n = np.arange(st.shape[0])
    assert (st[:, 0, 12] - r * st[:, 0, 16] > 0).all()  # contact point still slipping forward
    np.testing.assert_allclose(st[:, 0, 12], 3.0 - n * mu * G * h, rtol=1e-9)
    I, mass = float(m.inertia[0, 0, 1]), float(m.mass[0, 0])  # solid sphere: I = 2/5 m r^2
    np.testing.assert_allclose(st[:, 0, 16], n * mu * mass * G * h * r / I, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(st[:, 0, 2], r - m.slop, atol=1e-12)


def test_ball_contact_point_angular_momentum_invariant():
    """For a sphere centred on its body, every impulse (gravity, normal, friction, Baumgarte)
    passes through the vertical line of the centre, so L_c = I w + m (r z) x v is invariant
    through flight, impact, sliding and rolling; with e = 0 the final rolling speed is
    (5/7) of the initial horizontal speed (initial spin zero)."""
    m = WL.ball(B=4)
    r, mass = 0.1, 1.0
    I = 0.4 * mass * r * r
    for i in range(m.B):
        st, _, act, _ = O.rollout(m, i, log=True)
        assert act[:, 0].any()
        Lc = np.array([I * s[0, 15:18] + mass * np.cross([0.0, 0.0, r], s[0, 12:15]) for s in st])
        assert np.abs(Lc - Lc[0]).max() <= 1e-7 * np.linalg.norm(Lc[0])
        vh0 = m.state0[i, 0, 12:14]
        vf = st[-1, 0, 12:14]
        np.testing.assert_allclose(vf, 5.0 / 7.0 * vh0, rtol=1e-6, atol=1e-9)


def test_two_spheres_momentum_and_restitution():
    """Sphere-sphere contact: total linear momentum is exact; frictionless angular momentum
    about the origin is exact; with e = 0.5 the relative normal speed after the first contact
    step is -e times the one before (one row, solved exactly)."""
    m = WL.two_spheres(B=3, e=0.5, mu=0.0)
    m.slop = 0.1  # first-contact penetration stays inside the slop: no Baumgarte term
    masses = m.mass[0]
    pn = int(np.flatnonzero(O.schedule(m)["kind"] == 6)[0])  # the pair's normal row
    for i in range(m.B):
        st, _, act, gap = O.rollout(m, i, log=True)
        assert act[:, pn].any()
        P = st[:, 0, 12:15] * masses[0] + st[:, 1, 12:15] * masses[1]
        np.testing.assert_allclose(P, np.broadcast_to(P[0], P.shape), rtol=0, atol=1e-12)
        Ls = []
        for s in st:
            L = 0.0
            for b in range(2):
                R = s[b, 3:12].reshape(3, 3)
                Iw = R @ np.diag(m.inertia[i, b]) @ R.T
                L = L + Iw @ s[b, 15:18] + masses[b] * np.cross(s[b, 0:3], s[b, 12:15])
            Ls.append(L)
        Ls = np.array(Ls)
        assert np.abs(Ls - Ls[0]).max() <= 1e-9 * (1 + np.linalg.norm(Ls[0]))
        t = int(np.argmax(act[:, pn]))
        dx0 = st[t, 0, :3] - st[t, 1, :3]
        n = dx0 / np.linalg.norm(dx0)
        vn_before = (st[t, 0, 12:15] - st[t, 1, 12:15]) @ n
        vn_after = (st[t + 1, 0, 12:15] - st[t + 1, 1, 12:15]) @ n
        assert vn_before < 0
        depth = np.linalg.norm(dx0) - 0.25
        assert depth + m.slop >= 0  # only the restitution term acts in that step
        np.testing.assert_allclose(vn_after, -0.5 * vn_before, rtol=1e-10)


def test_free_body_invariants():
    """Asymmetric free body without gravity: linear momentum exact; Eq. 1 keeps R orthonormal;
    the explicit gyroscopic term drifts angular momentum and energy by O(h) (bounded here)."""
    m = WL.free_body(B=2, horizon=1000)
    for i in range(2):
        st, _, _, _ = O.rollout(m, i)
        np.testing.assert_allclose(st[:, 0, 12:15], np.broadcast_to(st[0, 0, 12:15], st[:, 0, 12:15].shape), atol=0)
        I = m.inertia[i, 0]

        def L_E(s):
            R = s[3:12].reshape(3, 3)
            Iw = R @ np.diag(I) @ R.T
            return Iw @ s[15:18], 0.5 * s[15:18] @ Iw @ s[15:18]

        L0, E0 = L_E(st[0, 0])
        LT, ET = L_E(st[-1, 0])
        assert np.linalg.norm(LT - L0) <= 5e-3 * np.linalg.norm(L0)
        assert abs(ET - E0) <= 5e-3 * E0
        for s in st[::50]:
            R = s[0, 3:12].reshape(3, 3)
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-9


def test_eq1_renormalisation_fixed_point_and_quadratic_contraction():
    """Eq. 1 (read as the polar step): a rotation is a fixed point, and the orthogonality
    error of a perturbed matrix shrinks quadratically (body at rest, no gravity)."""
    m = WL.free_body(B=1, horizon=1)
    x = m.state0[0].copy()
    x[0, 12:18] = 0.0
    R0 = np.array(WL._rot_z(0.7) @ WL._rot_y(-0.4))
    x[0, 3:12] = R0.reshape(9)
    xn, _, _, _ = O.step(m, 0, x)
    np.testing.assert_allclose(xn[0, 3:12], R0.reshape(9), atol=1e-15)
    E = np.random.default_rng(3).standard_normal((3, 3))
    errs = []
    for eps in (1e-2, 1e-3):
        x[0, 3:12] = (R0 + eps * E).reshape(9)
        xn, _, _, _ = O.step(m, 0, x)
        R = xn[0, 3:12].reshape(3, 3)
        errs.append(np.abs(R.T @ R - np.eye(3)).max())
    assert errs[1] < errs[0] / 50.0
    assert errs[0] < 1e-2 ** 2 * 20


def test_small_angle_pendulum_period():
    """Rod on a world hinge, 1 deg amplitude: period 2 pi sqrt(I_pivot / (m g d)), d = L/2."""
    L, mass, rr = 0.5, 1.0, 0.005
    m = WL.pendulum1(B=1, L=L, m=mass, amp_deg=1.0, horizon=3000, dt=0.001, rod_radius=rr)
    st, _, _, _ = O.rollout(m, 0)
    R = st[:, 0, 3:12].reshape(-1, 3, 3)
    ang = np.arctan2(R[:, 0, 2], R[:, 2, 2])
    t = np.arange(len(ang)) * m.dt
    zc = [t[k] - ang[k] * m.dt / (ang[k + 1] - ang[k]) for k in range(len(ang) - 1) if ang[k] > 0 >= ang[k + 1]]
    period = (zc[-1] - zc[0]) / (len(zc) - 1)
    Icm = mass * (3 * rr * rr + L * L) / 12.0
    T0 = 2 * math.pi * math.sqrt((Icm + mass * (L / 2) ** 2) / (mass * G * L / 2))
    assert abs(period - T0) / T0 < 2e-3


def test_three_link_chain_small_oscillation_frequencies():
    """3-link chain, small amplitude: the dominant frequency of the tip matches one of the
    normal-mode frequencies of the linearised chain (generalised eigenproblem K q = w^2 M q)."""
    rng = np.random.default_rng(5)
    m = WL.pendulum3(B=1, horizon=6000, dt=0.001, iters=20)
    Ls = m.link_length[0]
    masses = m.mass[0]
    Ic = m.inertia[0, :, 0]
    # initial pose: tiny angles, mostly along the first mode computed below
    n = 3
    # linearised mass and stiffness in absolute link angles phi_k
    Mm = np.zeros((n, n))
    Kk = np.zeros((n, n))
    for k in range(n):
        # centre of link k: sum_{j<k} L_j phi_j + L_k/2 phi_k (horizontal displacement)
        lever = np.zeros(n)
        for j in range(k):
            lever[j] = Ls[j]
        lever[k] = Ls[k] / 2
        Mm += masses[k] * np.outer(lever, lever)
        Mm[k, k] += Ic[k]
        Kk[k, k] += masses[k] * G * Ls[k] / 2
        for j in range(k):
            Kk[j, j] += masses[k] * G * Ls[j]
    from scipy.linalg import eigh
    w2, vecs = eigh(Kk, Mm)
    mode = vecs[:, 0] / np.abs(vecs[:, 0]).max() * math.radians(0.5)
    # rebuild the initial pose with relative angles from the mode's absolute angles
    rel = np.concatenate([[mode[0]], np.diff(mode)])
    phi, pivot = 0.0, np.zeros(3)
    for k in range(n):
        phi += rel[k]
        R = WL._rot_y(phi)
        m.state0[0, k] = WL._state(pivot + R @ np.array([0.0, 0.0, -Ls[k] / 2]), R, np.zeros(3), np.zeros(3))
        pivot = pivot + R @ np.array([0.0, 0.0, -Ls[k]])
    st, _, _, _ = O.rollout(m, 0)
    R0 = st[:, 0, 3:12].reshape(-1, 3, 3)
    ang = np.arctan2(R0[:, 0, 2], R0[:, 2, 2])
    t = np.arange(len(ang)) * m.dt
    zc = [t[k] - ang[k] * m.dt / (ang[k + 1] - ang[k]) for k in range(len(ang) - 1) if ang[k] > 0 >= ang[k + 1]]
    period = (zc[-1] - zc[0]) / (len(zc) - 1)
    T0 = 2 * math.pi / math.sqrt(w2[0])
    assert abs(period - T0) / T0 < 1e-2
    del rng


def test_chain_joint_drift_and_energy_bound():
    """Contact-free 3-link chains (h = 1 ms, 10 sweeps): joint separation stays below 1 mm over
    1000 steps, and total energy changes by less than 0.1 % of the chain's energy scale."""
    m = WL.pendulum3(B=4, horizon=1000)
    for i in range(m.B):
        st, _, _, _ = O.rollout(m, i)
        drift = 0.0
        for s in st[::10]:
            for j, (a, b) in enumerate(m.joint_body):
                pa = np.zeros(3) if a < 0 else s[a, :3]
                Ra = np.eye(3) if a < 0 else s[a, 3:12].reshape(3, 3)
                e = pa + Ra @ m.anchor[i, j, 0] - s[b, :3] - s[b, 3:12].reshape(3, 3) @ m.anchor[i, j, 1]
                drift = max(drift, np.linalg.norm(e))
        assert drift < 1e-3

        def energy(s):
            E = 0.0
            for b in range(3):
                R = s[b, 3:12].reshape(3, 3)
                E += 0.5 * m.mass[i, b] * s[b, 12:15] @ s[b, 12:15]
                E += 0.5 * s[b, 15:18] @ (R @ np.diag(m.inertia[i, b]) @ R.T) @ s[b, 15:18]
                E += m.mass[i, b] * G * s[b, 2]
            return E

        scale = sum(m.mass[i, b] * G * m.link_length[i].sum() for b in range(3))
        Es = np.array([energy(s) for s in st[::10]])
        assert np.abs(Es - Es[0]).max() < 1e-3 * scale


def test_servo_tracks_controller_output():
    """The controller's output is the servo's target angle: a rod on a motorised world hinge
    (no gravity, strong motor), fed a constant input (clock at 0 Hz -> (sin 0, cos 0)), settles
    at theta = u, where u is the dense network evaluated on the bfloat16-rounded input and
    weights (ReLU hidden layer, linear output)."""
    torch = pytest.importorskip("torch")
    m = WL.pendulum1(B=1, horizon=400, dt=0.005, iters=30)
    m.gravity = (0.0, 0.0, 0.0)
    m.joint_flags = np.array([WL.FLAG_MOTOR], np.int32)
    m.motor[0, 0] = [20.0, 100.0, 10.0]
    m.widths = [2, 16, 1]
    m.features = WL.F_CLOCK
    m.clock_hz = 0.0
    rng = np.random.default_rng(11)
    m.W = WL.xavier_weights(m.widths, 0, rng)
    m.W[2 * 16:2 * 16 + 16] = rng.uniform(-0.2, 0.2, 16).astype(np.float32)   # hidden biases
    m.W[-1] = np.float32(0.1)
    bf = lambda a: torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    W1 = bf(m.W[:32].reshape(16, 2))
    b1 = m.W[32:48].astype(np.float64)
    W2 = bf(m.W[48:64].reshape(1, 16))
    b2 = float(m.W[64])
    s = bf([0.0, 1.0])
    hdn = bf(np.maximum(W1 @ s + b1, 0.0))
    u = float((W2 @ hdn)[0]) + b2
    assert 0.05 < abs(u) < 1.5
    st, _, _, _ = O.rollout(m, 0)
    R = st[-1, 0, 3:12].reshape(3, 3)
    theta = math.atan2(R[0, 2], R[2, 2])
    assert abs(theta - u) < 1e-6


# ----------------------------------------------------------------------------- gradients
def _fd(fun, x0, idx, eps):
    out = []
    for k in idx:
        xp = x0.copy(); xp.flat[k] += eps
        xm = x0.copy(); xm.flat[k] -= eps
        out.append((fun(xp) - fun(xm)) / (2 * eps))
    return np.array(out)


def _same_activity(m, i, T, overrides_p, overrides_m, W_p=None, W_m=None):
    _, _, a1, _ = O.rollout(m, i, horizon=T, log=True, overrides=overrides_p, W=W_p)
    _, _, a2, _ = O.rollout(m, i, horizon=T, log=True, overrides=overrides_m, W=W_m)
    return np.array_equal(a1, a2)


def test_gradient_matches_central_differences_ball():
    """Ball through impact and sliding: reverse-mode gradient w.r.t. the initial velocity and
    spin, the radius and friction, equals central differences of the forward pass."""
    m = WL.ball(B=2, horizon=60)
    for i in range(m.B):
        m.state0[i, 0, 2] = 0.6
        m.state0[i, 0, 15:18] = [1.0, -2.0, 0.5]
        L, g = O.rollout_grad(m, i)
        checked = 0
        for key, idx in (("state0", [12, 13, 14, 15, 16]), ("sph_rad", [0]), ("sph_mu", [0])):
            base = getattr(m, key)[i].astype(np.float64)

            def f(v):
                return O.rollout(m, i, overrides={key: v})[1]

            eps = 1e-6
            for k in idx:
                xp = base.copy(); xp.flat[k] += eps
                xm = base.copy(); xm.flat[k] -= eps
                if not _same_activity(m, i, m.horizon, {key: xp}, {key: xm}):
                    continue
                fd = (f(xp) - f(xm)) / (2 * eps)
                assert abs(fd - g[key].flat[k]) <= 1e-5 * (abs(fd) + 1e-3), (key, k, fd, g[key].flat[k])
                checked += 1
        assert checked >= 5


def test_gradient_matches_central_differences_pendulum():
    """Contact-free 3-link chain, 80 steps: gradient w.r.t. anchors, inertia, masses and the
    initial state equals central differences."""
    m = WL.pendulum3(B=1, horizon=80)
    L, g = O.rollout_grad(m, 0)
    rng = np.random.default_rng(2)
    for key in ("anchor", "inertia", "mass", "state0"):
        base = getattr(m, key)[0].astype(np.float64)
        idx = rng.choice(base.size, size=min(6, base.size), replace=False)
        for k in idx:
            eps = 1e-6 * max(1.0, abs(base.flat[k]))
            xp = base.copy(); xp.flat[k] += eps
            xm = base.copy(); xm.flat[k] -= eps
            fd = (O.rollout(m, 0, overrides={key: xp})[1] - O.rollout(m, 0, overrides={key: xm})[1]) / (2 * eps)
            assert abs(fd - g[key].flat[k]) <= 2e-5 * (abs(fd) + 1e-2), (key, k, fd, g[key].flat[k])


def test_gradient_matches_central_differences_quadruped_controller():
    """Quadruped with the dense controller, 15 steps through ground contact, limits and motors:
    the reverse-mode gradient w.r.t. controller weights and the initial state equals central
    differences. bfloat16 rounding is piecewise constant, so this check runs the controller
    unrounded (the rounding's reverse mode is the identity, straight-through)."""
    m = WL.quadruped(B=1, horizon=15)
    m.exact_mlp = 1
    L, g = O.rollout_grad(m, 0)
    rng = np.random.default_rng(4)
    base = m.state0[0].astype(np.float64)
    checked = 0
    for k in rng.choice(base.size, 8, replace=False):
        eps = 1e-7
        xp = base.copy(); xp.flat[k] += eps
        xm = base.copy(); xm.flat[k] -= eps
        if not _same_activity(m, 0, m.horizon, {"state0": xp}, {"state0": xm}):
            continue
        fd = (O.rollout(m, 0, overrides={"state0": xp})[1] - O.rollout(m, 0, overrides={"state0": xm})[1]) / (2 * eps)
        assert abs(fd - g["state0"].flat[k]) <= 1e-4 * (abs(fd) + 1e-3), (k, fd, g["state0"].flat[k])
        checked += 1
    nb1 = 24 * 128
    for k in [0, 5, 77, 1000, nb1 + 3, nb1 + 50, nb1 + 128 + 999, len(m.W) - 20, len(m.W) - 3]:
        eps = 1e-6
        Wp = m.W.astype(np.float64).copy(); Wp[k] += eps
        Wm = m.W.astype(np.float64).copy(); Wm[k] -= eps
        if not _same_activity(m, 0, m.horizon, None, None, Wp, Wm):
            continue
        fd = (O.rollout(m, 0, W=Wp)[1] - O.rollout(m, 0, W=Wm)[1]) / (2 * eps)
        assert abs(fd - g["W"][k]) <= 1e-4 * (abs(fd) + 1e-4), (k, fd, g["W"][k])
        checked += 1
    assert checked >= 10


def test_gradient_decay_closed_form_in_flight():
    """Section 3.2's decay of the gradient by alpha per time step: for a ball in free flight the
    loss of the final position has dL/dv0 = T h alpha^(T-1) dL/dp_T (each step passes the
    adjoint of the later steps back scaled by alpha; T = 1 needs no decay)."""
    m = WL.ball(B=1, horizon=30)
    m.state0[0, 0, 2] = 5.0  # high enough not to land within 30 steps
    st, _, act, _ = O.rollout(m, 0, log=True)
    assert not act.any()
    g_pT = 2.0 * (st[-1, 0, :3] - m.loss_target[0])
    for alpha in (1.0, 0.9, 0.5):
        m.grad_decay = alpha
        _, g = O.rollout_grad(m, 0)
        np.testing.assert_allclose(g["state0"][0, 12:15], 30 * m.dt * alpha ** 29 * g_pT, rtol=1e-10)
        np.testing.assert_allclose(g["state0"][0, 0:3], alpha ** 29 * g_pT, rtol=1e-10)
