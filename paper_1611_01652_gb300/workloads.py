"""Seeded synthetic workloads: robot descriptions and initial states.

This module only *builds inputs*: body geometry, masses, inertias, joint frames, sphere
placements, initial poses and controller weights. It holds none of the stepping arithmetic
and is the one module that both the CUDA path and the FP64 oracle tests consume.

Every floating-point value is rounded to float32 before it is handed out (stored as float64
here), so the oracle and the GPU library read bit-identical inputs.

Workloads (the paper's experiments give their shapes; section numbers refer to the paper):
  * ``ball``       - one sphere thrown onto the ground (section 2.1.1 "Throwing a Ball").
  * ``pendulum3``  - contact-free 3-link hinge chains (shaped like the arm of section 3.2).
  * ``quadruped``  - box torso, 4 legs x 2 links on hinges with limits and servo motors,
                     sphere feet and 4 spheres inside the torso (section 3.1 and Fig. 3B),
                     driven by a dense controller (Eq. g).
  * ``two_spheres``- two free spheres colliding (sphere-sphere contact check).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

# Joint types, flags, feature bits and loss kinds (the same values are part of the C ABI).
BALL, HINGE = 0, 1
FLAG_LIMIT, FLAG_MOTOR = 1, 2
F_ANGLES, F_RATES, F_CLOCK, F_IMU, F_TARGET = 1, 2, 4, 8, 16
L_SQDIST, L_DIST, L_LINEAR, L_DISP = 0, 1, 2, 3
M_FINAL, M_MEAN = 0, 1


def f32(x):
    """Round to float32 and return float64 holding the same value."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Model:
    """A batch of robots that share one topology (one bin)."""

    name: str
    B: int
    # topology
    joint_type: np.ndarray
    joint_body: np.ndarray
    joint_flags: np.ndarray
    sphere_body: np.ndarray
    pair_sphere: np.ndarray
    nb: int
    # per-instance parameters, leading dimension B
    mass: np.ndarray
    inertia: np.ndarray
    anchor: np.ndarray
    axis: np.ndarray
    ref: np.ndarray
    limit: np.ndarray
    motor: np.ndarray
    sph_off: np.ndarray
    sph_rad: np.ndarray
    sph_mu: np.ndarray
    sph_e: np.ndarray
    loss_point: np.ndarray
    loss_target: np.ndarray
    state0: np.ndarray
    # controller
    widths: list = field(default_factory=list)
    skip: int = 0
    features: int = 0
    imu_body: int = 0
    clock_hz: float = 0.0
    W: np.ndarray | None = None
    # constants
    gravity: tuple = (0.0, 0.0, -9.81)
    dt: float = 0.01
    ground_z: float = 0.0
    beta: float = 0.2
    gamma: float = 0.0
    slop: float = 0.005
    iters: int = 20
    horizon: int = 100
    ckpt_every: int = 0
    loss_kind: int = L_SQDIST
    loss_mode: int = M_FINAL
    loss_body: int = 0
    ctrl_fp32: int = 0  # 1: controller without bfloat16 rounding (fp32 storage)

    @property
    def nj(self):
        return int(len(self.joint_type))

    @property
    def ns(self):
        return int(len(self.sphere_body))

    @property
    def np_(self):
        return int(len(self.pair_sphere))

    def subset(self, idx):
        """Instances ``idx`` of the batch as a new Model (shared topology/controller)."""
        idx = np.atleast_1d(np.asarray(idx))
        names = [f.name for f in dataclasses.fields(self)]
        kw = {k: getattr(self, k) for k in names}
        for k in PER_INSTANCE:
            kw[k] = getattr(self, k)[idx].copy()
        kw["B"] = int(len(idx))
        out = Model(**kw)
        for k, v in self.__dict__.items():
            if k in names:
                continue
            if isinstance(v, np.ndarray) and v.ndim > 0 and len(v) == self.B:
                setattr(out, k, v[idx].copy())  # per-instance extras (horizons, ids, ...)
            else:
                setattr(out, k, v)  # model-wide extras (gradient decay, ...)
        return out


PER_INSTANCE = ("mass", "inertia", "anchor", "axis", "ref", "limit", "motor", "sph_off", "sph_rad",
                "sph_mu", "sph_e", "loss_point", "loss_target", "state0")


def param_count(widths, skip=0):
    """Number of controller parameters: per dense layer W [out][in] and a bias [out];
    with ``skip`` the output layer also has a second biased dense layer from the input."""
    if not widths:
        return 0
    n = sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1))
    if skip:
        n += widths[0] * widths[-1] + widths[-1]
    return n


def xavier_weights(widths, skip, rng, zero_output=False, out_scale=1.0):
    """Flat float32 controller parameters: Xavier-uniform weights (the output layer, and the
    skip layer, scaled by ``out_scale``), zero biases."""
    parts = []
    L = len(widths) - 1
    for l in range(L):
        ni, no = widths[l], widths[l + 1]
        a = math.sqrt(6.0 / (ni + no))
        w = rng.uniform(-a, a, size=(no, ni))
        if l == L - 1:
            w *= 0.0 if zero_output else out_scale
        parts += [w.ravel(), np.zeros(no)]
    if skip:
        ni, no = widths[0], widths[-1]
        a = math.sqrt(6.0 / (ni + no))
        w = rng.uniform(-a, a, size=(no, ni)) * out_scale
        if zero_output:
            w[:] = 0.0
        parts += [w.ravel(), np.zeros(no)]
    return np.concatenate(parts).astype(np.float32) if parts else np.zeros(0, np.float32)


def _rot_z(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _rot_y(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _state(p, R, v, w):
    return np.concatenate([p, R.reshape(9), v, w])


def _empty(B, nb, nj, ns):
    return dict(
        mass=np.zeros((B, nb)), inertia=np.zeros((B, nb, 3)), anchor=np.zeros((B, nj, 2, 3)),
        axis=np.zeros((B, nj, 2, 3)), ref=np.zeros((B, nj, 2, 3)), limit=np.zeros((B, nj, 2)),
        motor=np.zeros((B, nj, 3)), sph_off=np.zeros((B, ns, 3)), sph_rad=np.zeros((B, ns)),
        sph_mu=np.zeros((B, ns)), sph_e=np.zeros((B, ns)), loss_point=np.zeros((B, 3)),
        loss_target=np.zeros((B, 3)), state0=np.zeros((B, nb, 18)))


def _finish(d):
    for k in PER_INSTANCE:
        d[k] = f32(d[k])
    return d


def ball(B=1, seed=1000, horizon=300, iters=20, dt=0.01):
    """Sphere r=0.1 m, m=1 kg, launched from the ground with speed U[2,8] m/s, elevation
    U[20,70] deg, azimuth U[0,2pi); ground friction 0.5, restitution 0. Loss: squared distance
    of the final centre to a seeded target point."""
    rng = np.random.default_rng(seed)
    d = _empty(B, 1, 0, 1)
    r, m = 0.1, 1.0
    d["mass"][:] = m
    d["inertia"][:] = 0.4 * m * r * r
    d["sph_rad"][:] = r
    d["sph_mu"][:] = 0.5
    d["sph_e"][:] = 0.0
    for i in range(B):
        sp = rng.uniform(2.0, 8.0)
        el = math.radians(rng.uniform(20.0, 70.0))
        az = rng.uniform(0.0, 2.0 * math.pi)
        v = sp * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        d["state0"][i, 0] = _state(np.array([0.0, 0.0, r]), np.eye(3), v, np.zeros(3))
        d["loss_target"][i] = [rng.uniform(-5, 5), rng.uniform(-5, 5), r]
    _finish(d)
    return Model(name="ball", B=B, joint_type=np.zeros(0, np.int32), joint_body=np.zeros((0, 2), np.int32),
                 joint_flags=np.zeros(0, np.int32), sphere_body=np.zeros(1, np.int32),
                 pair_sphere=np.zeros((0, 2), np.int32), nb=1, dt=dt, iters=iters, horizon=horizon,
                 loss_kind=L_SQDIST, loss_mode=M_FINAL, loss_body=0, **d)


def pendulum_sysid(B=4096, K=4, seed=1004, horizon=300, iters=10, dt=0.001, m0=1.0, rod_radius=0.02):
    """3-link pendulum chains for system identification of their link masses: B / K pendulums,
    each released K times from different seeded angles (instances g*K .. g*K+K-1 are the swings
    of pendulum g). Chains as ``pendulum3`` (lengths U[0.3,1.0] m, hinges about y, uniform-rod
    inertias of the nominal mass ``m0``), relative initial angles U[-pi/2, pi/2]. Each pendulum has
    hidden link masses ``mass_true`` U[0.5,2.0] kg (per instance, equal within a pendulum; the
    rotational inertias are the known nominal ones); the model starts from ``m0``. Loss: squared
    distance of the last link's far end at the final step to ``loss_target`` (its observed
    position, set by the caller)."""
    assert B % K == 0
    rng = np.random.default_rng(seed)
    nb = nj = 3
    d = _empty(B, nb, nj, 0)
    mass_true = np.zeros((B, nb))
    for g in range(B // K):
        L = rng.uniform(0.3, 1.0, size=nb)
        mt = rng.uniform(0.5, 2.0, size=nb)
        for i in range(g * K, (g + 1) * K):
            th = rng.uniform(-math.pi / 2, math.pi / 2, size=nb)
            phi = 0.0
            pivot = np.zeros(3)
            for k in range(nb):
                phi += th[k]
                R = _rot_y(phi)
                c = pivot + R @ np.array([0.0, 0.0, -L[k] / 2])
                d["state0"][i, k] = _state(c, R, np.zeros(3), np.zeros(3))
                pivot = pivot + R @ np.array([0.0, 0.0, -L[k]])
                d["mass"][i, k] = m0
                It = m0 * (3 * rod_radius ** 2 + L[k] ** 2) / 12.0
                d["inertia"][i, k] = [It, It, 0.5 * m0 * rod_radius ** 2]
                d["anchor"][i, k, 0] = [0.0, 0.0, 0.0] if k == 0 else [0.0, 0.0, -L[k - 1] / 2]
                d["anchor"][i, k, 1] = [0.0, 0.0, L[k] / 2]
                d["axis"][i, k, :] = [0.0, 1.0, 0.0]
                d["ref"][i, k, :] = [1.0, 0.0, 0.0]
            d["loss_point"][i] = [0.0, 0.0, -L[2] / 2]
            mass_true[i] = mt
    _finish(d)
    mdl = Model(name="pendulum_sysid", B=B, joint_type=np.full(nj, HINGE, np.int32),
                joint_body=np.array([[-1, 0], [0, 1], [1, 2]], np.int32), joint_flags=np.zeros(nj, np.int32),
                sphere_body=np.zeros(0, np.int32), pair_sphere=np.zeros((0, 2), np.int32), nb=nb, dt=dt,
                iters=iters, horizon=horizon, loss_kind=L_SQDIST, loss_mode=M_FINAL, loss_body=2, **d)
    mdl.mass_true = f32(mass_true)
    mdl.throws = K
    return mdl


class CameraScene:
    """A camera looking at textured objects carried by a model's bodies (attributes: W, H, f (focal
    length in pixels), plane (distance of the projection plane, m), cam_pos [3], cam_rot [3, 3] (rows: image right, image down, optical axis), obj_body,
    obj_center [n, 3], obj_half [n, 3], obj_tex, textures [n_tex, th, tw, 3], states [B, nb, 18],
    and optionally obj_kind [n]: 0 box, 1 sphere of radius half[0], 2 plane; absent: all boxes)."""


def procedural_textures(n, th=64, tw=64, seed=7):
    """Seeded smooth colour patterns (sums of a few random plane waves plus a checker), values in
    [0, 1]: stand-ins for the photographs the paper's textures were made from."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid((np.arange(th) + 0.5) / th, (np.arange(tw) + 0.5) / tw, indexing="ij")
    out = np.zeros((n, th, tw, 3), np.float32)
    for t in range(n):
        for ch in range(3):
            v = np.full((th, tw), 0.5)
            for _ in range(3):
                kx, ky, ph = rng.uniform(-8, 8), rng.uniform(-8, 8), rng.uniform(0, 2 * math.pi)
                v += 0.15 * np.sin(2 * math.pi * (kx * xx + ky * yy) + ph)
            v += 0.1 * np.sign(np.sin(2 * math.pi * 4 * xx) * np.sin(2 * math.pi * 4 * yy))
            out[t, :, :, ch] = np.clip(v, 0.0, 1.0)
    return out


def camera_scene(B=4096, W=288, H=96, seed=1005, tex_size=64, mixed=False):
    """The 3-link pendulum seen by a camera (the paper's camera sensor, section 3.4, at its 288 x 96
    resolution): the three links as textured boxes (0.12 x 0.12 x L m) on bodies 0-2, a textured
    backdrop box 1 m behind the hinge plane, and a camera 3 m in front of it looking along +y
    (image right = +x, image down = -z), focal length W / 2 pixels, projection plane 0.05 m in
    front of it. With ``mixed`` also a sphere of radius 0.09 m at the far end of the last link and
    a textured ground plane 1.5 m below the hinge (texture period 1 m). States: ``pendulum3``
    chains (seeded lengths and angles), positions only."""
    pm = pendulum3(B=B, seed=seed, horizon=1)
    cs = CameraScene()
    cs.W, cs.H, cs.f, cs.plane = W, H, 0.5 * W, 0.05
    cs.cam_pos = np.array([0.0, -3.0, -0.9])
    cs.cam_rot = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
    L = pm.link_length[0]
    cs.obj_body = np.array([-1, 0, 1, 2], np.int32)
    cs.obj_center = np.array([[0.0, 1.0, -0.9], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    cs.obj_half = np.array([[8.0, 0.05, 3.0], [0.06, 0.06, L[0] / 2], [0.06, 0.06, L[1] / 2], [0.06, 0.06, L[2] / 2]])
    cs.obj_tex = np.array([0, 1, 2, 3], np.int32)
    cs.textures = procedural_textures(4, tex_size, tex_size, seed)
    if mixed:
        cs.obj_body = np.concatenate([cs.obj_body, [2, -1]]).astype(np.int32)
        cs.obj_center = np.concatenate([cs.obj_center, [[0.0, 0.0, -L[2] / 2], [0.0, 0.0, -1.5]]])
        cs.obj_half = np.concatenate([cs.obj_half, [[0.09, 0.09, 0.09], [0.5, 0.5, 1.0]]])
        cs.obj_tex = np.array([0, 1, 2, 3, 4, 5], np.int32)
        cs.obj_kind = np.array([0, 0, 0, 0, 1, 2], np.int32)
        cs.textures = procedural_textures(6, tex_size, tex_size, seed)
    st = np.asarray(pm.state0, np.float32).copy()
    # every instance carries the first chain's link lengths (the boxes are shared); its own angles
    for i in range(B):
        R = [st[i, k, 3:12].reshape(3, 3) for k in range(3)]
        pivot = np.zeros(3)
        for k in range(3):
            st[i, k, 0:3] = pivot + R[k] @ np.array([0.0, 0.0, -L[k] / 2])
            pivot = pivot + R[k] @ np.array([0.0, 0.0, -L[k]])
    cs.states = st
    cs.nb = 3
    return cs


def pendulum3(B=1024, seed=1001, horizon=1000, iters=10, dt=0.001, ckpt_every=32, rod_radius=0.02):
    """3-link pendulum chains, first hinge pinned to the world at the origin, horizontal (y)
    hinge axes. Links are uniform rods (thin cylinders of radius ``rod_radius``) of length
    U[0.3,1.0] m and mass U[0.5,2.0] kg; relative initial angles U[-pi/2, pi/2]. Loss: height
    of the far end of the last link at the final step."""
    rng = np.random.default_rng(seed)
    nb = nj = 3
    d = _empty(B, nb, nj, 0)
    Ls = np.zeros((B, nb))
    for i in range(B):
        L = rng.uniform(0.3, 1.0, size=nb)
        m = rng.uniform(0.5, 2.0, size=nb)
        th = rng.uniform(-math.pi / 2, math.pi / 2, size=nb)
        Ls[i] = L
        phi = 0.0
        pivot = np.zeros(3)
        for k in range(nb):
            phi += th[k]
            R = _rot_y(phi)
            c = pivot + R @ np.array([0.0, 0.0, -L[k] / 2])
            d["state0"][i, k] = _state(c, R, np.zeros(3), np.zeros(3))
            pivot = pivot + R @ np.array([0.0, 0.0, -L[k]])
            d["mass"][i, k] = m[k]
            It = m[k] * (3 * rod_radius ** 2 + L[k] ** 2) / 12.0
            d["inertia"][i, k] = [It, It, 0.5 * m[k] * rod_radius ** 2]
            d["anchor"][i, k, 0] = [0.0, 0.0, 0.0] if k == 0 else [0.0, 0.0, -L[k - 1] / 2]
            d["anchor"][i, k, 1] = [0.0, 0.0, L[k] / 2]
            d["axis"][i, k, :] = [0.0, 1.0, 0.0]
            d["ref"][i, k, :] = [1.0, 0.0, 0.0]
        d["loss_point"][i] = [0.0, 0.0, -L[2] / 2]
        d["loss_target"][i] = [0.0, 0.0, 1.0]
    _finish(d)
    mdl = Model(name="pendulum3", B=B, joint_type=np.full(nj, HINGE, np.int32),
                joint_body=np.array([[-1, 0], [0, 1], [1, 2]], np.int32), joint_flags=np.zeros(nj, np.int32),
                sphere_body=np.zeros(0, np.int32), pair_sphere=np.zeros((0, 2), np.int32), nb=nb, dt=dt,
                iters=iters, horizon=horizon, ckpt_every=ckpt_every, loss_kind=L_LINEAR, loss_mode=M_FINAL,
                loss_body=2, **d)
    mdl.link_length = f32(Ls)
    return mdl


def _capsule_inertia(m, r, L):
    """Principal moments of a solid capsule (cylinder of length L and radius r along z plus two
    hemispherical caps), total mass m."""
    vc = math.pi * r * r * L
    vs = 4.0 / 3.0 * math.pi * r ** 3
    mc, ms = m * vc / (vc + vs), m * vs / (vc + vs)
    Iz = mc * r * r / 2 + ms * 2 * r * r / 5
    Ix = mc * (L * L / 12 + r * r / 4) + ms * (2 * r * r / 5 + L * L / 4 + 3 * L * r / 8)
    return [Ix, Ix, Iz]


QUADRUPED_WIDTHS = [24, 128, 128, 8]


def quadruped(B=4096, seed=1002, horizon=1000, iters=20, dt=0.01, widths=None, skip=0, yaw=0.3, vel=0.1,
              w_seed=None, out_scale=0.1, n_recurrent=0):
    """Quadruped: box torso 0.6x0.3x0.1 m, 8 kg; 4 legs x 2 capsule links (0.2 m, radius 0.025,
    0.5 kg) on hinges about the body y axis with limits +-60 deg and servo motors (gain 30 1/s,
    4 N m, 45 deg/s); sphere feet r=0.03 and four r=0.05 spheres inside the torso, all touching
    the ground with mu=0.8, e=0. Hips at the torso corners. Dense controller
    24->128->128->8 (Xavier-uniform, seeded) fed by 8 joint angles, 8 joint rates, a
    1.5 Hz sin/cos clock and the torso's gravity direction and angular rate (body frame).
    Loss: negative forward (x) displacement of the torso. Per instance a seeded yaw in
    [-yaw, yaw] and a common horizontal velocity in [-vel, vel]^2.

    ``n_recurrent`` = H > 0 gives the controller the recurrent state of Eq. g: the network
    (default 24+H -> 128 -> 128 -> 8+H) reads the sensors and h^t, and its last H outputs give
    h^{t+1} = tanh(.), starting from h^0 = 0.

    The output layer's Xavier weights are scaled by ``out_scale`` (0.1): the paper starts its
    quadruped controller from a zero output layer (section 3.3); a full-size random output layer
    closes an unstable feedback loop through the servos (gain 30/s) whose reverse-mode gradient
    grows about e^0.24 per step and overflows float32 within a few hundred steps."""
    rng = np.random.default_rng(seed)
    if widths is None and n_recurrent:
        widths = [QUADRUPED_WIDTHS[0] + n_recurrent, *QUADRUPED_WIDTHS[1:-1], QUADRUPED_WIDTHS[-1] + n_recurrent]
    widths = list(widths or QUADRUPED_WIDTHS)
    nb, nj, ns = 9, 8, 8
    d = _empty(B, nb, nj, ns)
    hips = [(0.3, 0.15), (0.3, -0.15), (-0.3, 0.15), (-0.3, -0.15)]
    link, crad, cm = 0.2, 0.025, 0.5
    foot_r, torso_r = 0.03, 0.05
    z0 = 2 * link + foot_r - 0.001  # feet start 1 mm inside the ground (inside the slop)
    jt = np.full(nj, HINGE, np.int32)
    jb = np.zeros((nj, 2), np.int32)
    jf = np.full(nj, FLAG_LIMIT | FLAG_MOTOR, np.int32)
    sb = np.zeros(ns, np.int32)
    # local body poses at yaw 0 (body frame axes aligned with the world)
    local = [np.array([0.0, 0.0, z0])]
    for l, (hx, hy) in enumerate(hips):
        local.append(np.array([hx, hy, z0 - link / 2]))
        local.append(np.array([hx, hy, z0 - 1.5 * link]))
        jb[2 * l] = [0, 1 + 2 * l]
        jb[2 * l + 1] = [1 + 2 * l, 2 + 2 * l]
        sb[l] = 2 + 2 * l
        sb[4 + l] = 0
    I_torso = [8.0 / 12 * (0.3 ** 2 + 0.1 ** 2), 8.0 / 12 * (0.6 ** 2 + 0.1 ** 2), 8.0 / 12 * (0.6 ** 2 + 0.3 ** 2)]
    I_link = _capsule_inertia(cm, crad, link)
    for i in range(B):
        psi = rng.uniform(-yaw, yaw)
        vxy = rng.uniform(-vel, vel, size=2)
        Rz = _rot_z(psi)
        c0 = local[0]
        for b in range(nb):
            p = c0 + Rz @ (local[b] - c0)
            d["state0"][i, b] = _state(p, Rz, np.array([vxy[0], vxy[1], 0.0]), np.zeros(3))
        d["mass"][i, 0] = 8.0
        d["inertia"][i, 0] = I_torso
        d["mass"][i, 1:] = cm
        d["inertia"][i, 1:] = I_link
        for l, (hx, hy) in enumerate(hips):
            d["anchor"][i, 2 * l, 0] = [hx, hy, 0.0]
            d["anchor"][i, 2 * l, 1] = [0.0, 0.0, link / 2]
            d["anchor"][i, 2 * l + 1, 0] = [0.0, 0.0, -link / 2]
            d["anchor"][i, 2 * l + 1, 1] = [0.0, 0.0, link / 2]
            d["sph_off"][i, l] = [0.0, 0.0, -link / 2]
            d["sph_rad"][i, l] = foot_r
            d["sph_off"][i, 4 + l] = [0.25 * np.sign(hx), 0.1 * np.sign(hy), 0.0]
            d["sph_rad"][i, 4 + l] = torso_r
        d["axis"][i, :, :] = [0.0, 1.0, 0.0]
        d["ref"][i, :, :] = [1.0, 0.0, 0.0]
        d["limit"][i, :] = [-math.pi / 3, math.pi / 3]
        d["motor"][i, :] = [30.0, 4.0, math.pi / 4]
        d["sph_mu"][i] = 0.8
        d["sph_e"][i] = 0.0
        d["loss_point"][i] = [0.0, 0.0, 0.0]
        d["loss_target"][i] = [-1.0, 0.0, 0.0]
    _finish(d)
    wr = np.random.default_rng(seed + 7 if w_seed is None else w_seed)
    W = xavier_weights(widths, skip, wr, out_scale=out_scale)
    m = Model(name="quadruped", B=B, joint_type=jt, joint_body=jb, joint_flags=jf, sphere_body=sb,
              pair_sphere=np.zeros((0, 2), np.int32), nb=nb, widths=widths, skip=skip,
              features=F_ANGLES | F_RATES | F_CLOCK | F_IMU, imu_body=0, clock_hz=1.5, W=W, dt=dt,
              iters=iters, horizon=horizon, loss_kind=L_DISP, loss_mode=M_FINAL, loss_body=0, **d)
    m.n_recurrent = int(n_recurrent)
    return m


def two_spheres(B=4, seed=1003, horizon=60, iters=20, dt=0.01, e=0.0, mu=0.3, gravity=(0.0, 0.0, 0.0)):
    """Two free spheres (r=0.1 and 0.15 m, masses 1 and 2 kg) flying at each other above the
    ground (zero gravity by default), one sphere-sphere candidate pair. Loss: squared distance
    of sphere 0's centre to a target."""
    rng = np.random.default_rng(seed)
    nb, ns = 2, 2
    d = _empty(B, nb, 0, ns)
    for i in range(B):
        r = np.array([0.1, 0.15])
        m = np.array([1.0, 2.0])
        d["mass"][i] = m
        d["inertia"][i, 0] = 0.4 * m[0] * r[0] ** 2
        d["inertia"][i, 1] = 0.4 * m[1] * r[1] ** 2
        d["sph_rad"][i] = r
        d["sph_mu"][i] = mu
        d["sph_e"][i] = e
        off = rng.uniform(-0.08, 0.08, size=2)
        dz = rng.uniform(0.04, 0.1) * rng.choice([-1.0, 1.0])  # off-axis impact: normals away from n_z = 0
        p0 = np.array([-0.6, off[0], 1.0])
        p1 = np.array([0.6, off[1], 1.0 + dz])
        v0 = np.array([rng.uniform(2.0, 4.0), 0.0, 0.0])
        v1 = np.array([-rng.uniform(1.0, 3.0), 0.0, 0.0])
        w0 = rng.uniform(-2, 2, size=3)
        w1 = rng.uniform(-2, 2, size=3)
        d["state0"][i, 0] = _state(p0, np.eye(3), v0, w0)
        d["state0"][i, 1] = _state(p1, np.eye(3), v1, w1)
        d["loss_target"][i] = [0.0, 0.0, 1.0]
    _finish(d)
    return Model(name="two_spheres", B=B, joint_type=np.zeros(0, np.int32), joint_body=np.zeros((0, 2), np.int32),
                 joint_flags=np.zeros(0, np.int32), sphere_body=np.array([0, 1], np.int32),
                 pair_sphere=np.array([[0, 1]], np.int32), nb=nb, gravity=tuple(gravity), dt=dt, iters=iters,
                 horizon=horizon, ground_z=-10.0, loss_kind=L_SQDIST, loss_mode=M_FINAL, loss_body=0, **d)


def free_body(B=2, seed=1004, horizon=200, dt=0.001, iters=1):
    """One asymmetric free box without gravity or contacts, spinning about a seeded axis."""
    rng = np.random.default_rng(seed)
    d = _empty(B, 1, 0, 0)
    for i in range(B):
        d["mass"][i] = 2.0
        d["inertia"][i, 0] = [0.1, 0.2, 0.3]
        d["state0"][i, 0] = _state(rng.uniform(-1, 1, 3), np.eye(3), rng.uniform(-1, 1, 3), rng.uniform(-3, 3, 3))
        d["loss_target"][i] = [1.0, 2.0, 3.0]
    _finish(d)
    return Model(name="free_body", B=B, joint_type=np.zeros(0, np.int32), joint_body=np.zeros((0, 2), np.int32),
                 joint_flags=np.zeros(0, np.int32), sphere_body=np.zeros(0, np.int32),
                 pair_sphere=np.zeros((0, 2), np.int32), nb=1, gravity=(0.0, 0.0, 0.0), dt=dt, iters=iters,
                 horizon=horizon, loss_kind=L_SQDIST, loss_mode=M_FINAL, loss_body=0, **d)


def pendulum1(B=1, L=0.5, m=1.0, amp_deg=1.0, horizon=3000, dt=0.001, iters=20, rod_radius=0.005):
    """Single rod on a world hinge, released from a small angle (period check)."""
    d = _empty(B, 1, 1, 0)
    th = math.radians(amp_deg)
    R = _rot_y(th)
    for i in range(B):
        d["state0"][i, 0] = _state(R @ np.array([0.0, 0.0, -L / 2]), R, np.zeros(3), np.zeros(3))
        d["mass"][i] = m
        It = m * (3 * rod_radius ** 2 + L ** 2) / 12.0
        d["inertia"][i, 0] = [It, It, 0.5 * m * rod_radius ** 2]
        d["anchor"][i, 0, 0] = [0.0, 0.0, 0.0]
        d["anchor"][i, 0, 1] = [0.0, 0.0, L / 2]
        d["axis"][i, 0] = [0.0, 1.0, 0.0]
        d["ref"][i, 0] = [1.0, 0.0, 0.0]
        d["loss_point"][i] = [0.0, 0.0, -L / 2]
        d["loss_target"][i] = [0.0, 0.0, 1.0]
    _finish(d)
    return Model(name="pendulum1", B=B, joint_type=np.array([HINGE], np.int32), joint_body=np.array([[-1, 0]], np.int32),
                 joint_flags=np.zeros(1, np.int32), sphere_body=np.zeros(0, np.int32),
                 pair_sphere=np.zeros((0, 2), np.int32), nb=1, dt=dt, iters=iters, horizon=horizon,
                 loss_kind=L_LINEAR, loss_mode=M_FINAL, loss_body=0, **d)


ARM_WIDTHS = [32, 256, 256, 7]


ARM4_WIDTHS = [11, 64, 64, 4]


def arm4dof(B=256, seed=1006, horizon=300, iters=20, dt=0.005, widths=None, grad_decay=0.5, w_seed=None,
            bend=(0.5, 1.0)):
    """The paper's 4-degree-of-freedom arm (section 3.2): 1 m long, 32 kg, a 2-DoF actuated
    universal joint at the base and another at the elbow, servos of gain 30 1/s, 30 N m and
    45 deg/s. A universal (Cardan) joint is two revolute joints whose perpendicular axes meet in
    one point; here each is a hinge pair with a cross body (2 kg, moments of inertia 0.1 kg m^2,
    a motor housing; lighter crosses let the 20 sweeps leave the hinges drifting by centiradians)
    between them: the base cross yaws about the world z axis and the upper arm pitches about the
    cross's y axis; at the elbow the cross pitches about the upper arm's y axis and the forearm
    rolls about the cross's x axis. Upper arm and forearm: 0.5 m, 14 kg each (uniform rods, radius
    0.04 m); steps of 5 ms. The arm starts at rest with its base at the origin, the upper arm
    pitched by ``bend[0]`` and the elbow by ``bend[1]`` rad (upright, (0, 0), is a kinematic
    singularity: the tip lies on the base yaw axis); the hinges' reference vectors make that
    pose the zero of every joint angle, so the zero policy holds it. No gravity (with 30 N m the servos cannot hold
    32 kg of arm off the vertical). Per instance a seeded target at 0.3-0.9 m from the base in the
    upper half-space. Controller 11 -> 64 -> 64 -> 4 fed by the 4 joint angles and rates and the
    tip-to-target vector, its output layer zero (the paper starts from the zero policy). Loss: the
    tip's distance to the target averaged over the steps (the paper's per-step averaged
    objective), reverse mode with the gradient decay ``grad_decay`` (section 3.2; 0.5: at 0.9 the
    servo feedback loop of a trained controller makes the gradient grow to 1e40 within a few
    dozen training iterations on the FP64 oracle)."""
    rng = np.random.default_rng(seed)
    widths = list(widths or ARM4_WIDTHS)
    nb = nj = 4
    d = _empty(B, nb, nj, 0)
    Lk, mk, rk = 0.5, 14.0, 0.04
    It = mk * (3 * rk ** 2 + Lk ** 2) / 12.0
    mc, Ic = 2.0, 0.1
    R1 = _rot_y(bend[0])
    R2 = R1 @ _rot_y(bend[1])
    elbow = R1 @ np.array([0.0, 0.0, 0.5])
    poses = [(np.zeros(3), np.eye(3)), (R1 @ np.array([0.0, 0.0, 0.25]), R1), (elbow, R2),
             (elbow + R2 @ np.array([0.0, 0.0, 0.25]), R2)]
    ref_up = _rot_y(-bend[0]) @ np.array([1.0, 0.0, 0.0])  # x of the cross, seen from the upper arm
    ref_el = _rot_y(-bend[1]) @ np.array([1.0, 0.0, 0.0])  # x of the upper arm, seen from the elbow cross
    for i in range(B):
        # bodies: 0 base cross at the origin, 1 upper arm, 2 elbow cross, 3 forearm
        for k, (c, R) in enumerate(poses):
            d["state0"][i, k] = _state(c, R, np.zeros(3), np.zeros(3))
        d["mass"][i] = [mc, mk, mc, mk]
        d["inertia"][i] = [[Ic, Ic, Ic], [It, It, 0.5 * mk * rk ** 2], [Ic, Ic, Ic], [It, It, 0.5 * mk * rk ** 2]]
        d["anchor"][i, 0] = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]
        d["anchor"][i, 1] = [[0.0, 0.0, 0.0], [0.0, 0.0, -0.25]]
        d["anchor"][i, 2] = [[0.0, 0.0, 0.25], [0.0, 0.0, 0.0]]
        d["anchor"][i, 3] = [[0.0, 0.0, 0.0], [0.0, 0.0, -0.25]]
        d["axis"][i, 0] = [[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]]
        d["ref"][i, 0] = [[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
        d["axis"][i, 1] = [[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]
        d["ref"][i, 1] = [[1.0, 0.0, 0.0], ref_up]
        d["axis"][i, 2] = [[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]
        d["ref"][i, 2] = [[1.0, 0.0, 0.0], ref_el]
        d["axis"][i, 3] = [[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
        d["ref"][i, 3] = [[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]
        d["motor"][i, :] = [30.0, 30.0, math.pi / 4]
        d["limit"][i, :] = [-math.pi, math.pi]
        rr = rng.uniform(0.3, 0.9)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        u[2] = abs(u[2])
        d["loss_point"][i] = [0.0, 0.0, 0.25]
        d["loss_target"][i] = rr * u
    _finish(d)
    wr = np.random.default_rng(seed + 7 if w_seed is None else w_seed)
    W = xavier_weights(widths, 0, wr, zero_output=True)
    mdl = Model(name="arm4dof", B=B, joint_type=np.full(nj, HINGE, np.int32),
                joint_body=np.array([[-1, 0], [0, 1], [1, 2], [2, 3]], np.int32),
                joint_flags=np.full(nj, FLAG_MOTOR, np.int32), sphere_body=np.zeros(0, np.int32),
                pair_sphere=np.zeros((0, 2), np.int32), nb=nb, widths=widths, features=F_ANGLES | F_RATES | F_TARGET,
                W=W, dt=dt, iters=iters, horizon=horizon, loss_kind=L_DIST, loss_mode=M_MEAN, loss_body=3,
                gravity=(0.0, 0.0, 0.0), **d)
    mdl.grad_decay = grad_decay
    return mdl


def arms(B=8192, seed=1003, iters=10, dt=0.005, hmin=200, hmax=2000, links=(3, 7), widths=None, out_scale=0.1,
         w_seed=None, tau_max=60.0, grad_decay=0.9):
    """Uneven batch of robot arms on a table, returned as one Model per link count (a bin of one
    topology), each with per-instance ``horizons`` and the instances' original indices ``ids``.

    Per instance: n ~ U{links} hinged links (capsules of radius 0.02 m, length U[0.1, 0.4] m, mass
    2 kg/m x length) stacked upward from a base 0.1 m above the table (z = 0); joint 0 yaws about
    the world z axis (motor only), the other joints pitch about their body y axes (limits
    +-0.75 pi, motors); servos gain 10 1/s, ``tau_max`` N m (60 N m holds the longest arm, six
    0.4 m links, level against gravity: 56.5 N m; weaker servos let long arms collapse into
    chaotic swinging whose reverse-mode gradient overflows), 90 deg/s. A sphere of radius 0.03 m
    at the tip (mu 0.5, e 0) touches the table. Initial yaw U[-pi, pi], relative pitches
    U[-0.6, 0.6], at rest. Horizon U{hmin..hmax} steps of 5 ms. Controller 32 -> 256 -> 256 -> 7
    (bfloat16; 76,039 parameters, Xavier-uniform, output layer x ``out_scale``) shared by all
    instances, fed by the n joint angles, n joint rates and the tip-to-target vector (zero padded
    to 32); outputs beyond n are unused. Loss: distance of the tip to a seeded target on or above
    the table at the instance's last step. Reverse mode decays the gradient by ``grad_decay`` per
    step (section 3.2): over horizons of up to 2000 steps a few long arms still swing chaotically,
    and without the decay their gradients exceed the float32 range (1e32 for one 7-link arm over
    1302 steps on the FP64 oracle; 6e14 with alpha = 0.97). With alpha = 0.9 (a memory of about
    ten steps, 50 ms) every arm's gradient stays finite in float32."""
    rng = np.random.default_rng(seed)
    widths = list(widths or ARM_WIDTHS)
    n_of = rng.integers(links[0], links[1] + 1, size=B)
    h_of = rng.integers(hmin, hmax + 1, size=B)
    base_z, crad, tip_r = 0.1, 0.02, 0.03
    per = []
    for i in range(B):
        n = int(n_of[i])
        L = rng.uniform(0.1, 0.4, size=n)
        psi = rng.uniform(-math.pi, math.pi)
        th = rng.uniform(-0.6, 0.6, size=n)
        th[0] = 0.0
        reach = float(L.sum())
        rr = rng.uniform(0.2, 0.8) * reach
        ang = rng.uniform(0.0, 2.0 * math.pi)
        target = np.array([rr * math.cos(ang), rr * math.sin(ang), rng.uniform(0.03, 0.3)])
        per.append((n, L, psi, th, target))
    wr = np.random.default_rng(seed + 7 if w_seed is None else w_seed)
    W = xavier_weights(widths, 0, wr, out_scale=out_scale)
    bins = {}
    for n in range(links[0], links[1] + 1):
        ids = np.flatnonzero(n_of == n)
        if len(ids) == 0:
            continue
        Bn = len(ids)
        d = _empty(Bn, n, n, 1)
        for r, i in enumerate(ids):
            _, L, psi, th, target = per[i]
            pivot = np.array([0.0, 0.0, base_z])
            pitch = 0.0
            for k in range(n):
                pitch += th[k]
                R = _rot_z(psi) @ _rot_y(pitch)
                c = pivot + R @ np.array([0.0, 0.0, L[k] / 2])
                d["state0"][r, k] = _state(c, R, np.zeros(3), np.zeros(3))
                pivot = pivot + R @ np.array([0.0, 0.0, L[k]])
                d["mass"][r, k] = 2.0 * L[k]
                d["inertia"][r, k] = _capsule_inertia(2.0 * L[k], crad, L[k])
                d["anchor"][r, k, 0] = [0.0, 0.0, base_z] if k == 0 else [0.0, 0.0, L[k - 1] / 2]
                d["anchor"][r, k, 1] = [0.0, 0.0, -L[k] / 2]
                d["axis"][r, k, :] = [0.0, 0.0, 1.0] if k == 0 else [0.0, 1.0, 0.0]
                d["ref"][r, k, :] = [1.0, 0.0, 0.0]
                d["limit"][r, k] = [-0.75 * math.pi, 0.75 * math.pi]
                d["motor"][r, k] = [10.0, tau_max, math.pi / 2]
            d["sph_off"][r, 0] = [0.0, 0.0, L[n - 1] / 2]
            d["sph_rad"][r, 0] = tip_r
            d["sph_mu"][r, 0] = 0.5
            d["sph_e"][r, 0] = 0.0
            d["loss_point"][r] = [0.0, 0.0, L[n - 1] / 2]
            d["loss_target"][r] = target
        _finish(d)
        jb = np.array([[k - 1, k] for k in range(n)], np.int32)
        jf = np.array([FLAG_MOTOR] + [FLAG_LIMIT | FLAG_MOTOR] * (n - 1), np.int32)
        hz = h_of[ids].astype(np.int32)
        mdl = Model(name="arm%d" % n, B=Bn, joint_type=np.full(n, HINGE, np.int32), joint_body=jb, joint_flags=jf,
                    sphere_body=np.array([n - 1], np.int32), pair_sphere=np.zeros((0, 2), np.int32), nb=n,
                    widths=widths, features=F_ANGLES | F_RATES | F_TARGET, W=W, dt=dt, iters=iters,
                    horizon=int(hz.max()), loss_kind=L_DIST, loss_mode=M_FINAL, loss_body=n - 1, **d)
        mdl.horizons = hz
        mdl.ids = ids.astype(np.int64)
        mdl.grad_decay = grad_decay
        bins[n] = mdl
    return bins
