"""ctypes binding of the FP64 CPU oracle (``dp_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``; never by the library. It takes the plain numpy arrays of a
workload description (any object with the attributes of ``workloads.Model``) and never
touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dp_oracle.cpp")
LIB = os.path.join(HERE, "_build", "liboracle.so")


def build(force=False):
    """Compile the oracle with the host C++ compiler (plain IEEE FP64, no fast-math)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_bf16.restype = C.c_double
        _lib.orc_bf16.argtypes = [C.c_double]
    return _lib


PI = C.POINTER(C.c_int32)
PD = C.POINTER(C.c_double)


class Topo(C.Structure):
    _fields_ = [("nb", C.c_int32), ("nj", C.c_int32), ("ns", C.c_int32), ("np", C.c_int32),
                ("joint_type", PI), ("joint_body", PI), ("joint_flags", PI), ("sphere_body", PI),
                ("pair_sphere", PI), ("n_layers", C.c_int32), ("widths", PI), ("skip", C.c_int32),
                ("features", C.c_int32), ("imu_body", C.c_int32), ("clock_hz", C.c_double),
                ("gravity", C.c_double * 3), ("dt", C.c_double), ("ground_z", C.c_double),
                ("beta", C.c_double), ("gamma", C.c_double), ("slop", C.c_double), ("iters", C.c_int32),
                ("loss_kind", C.c_int32), ("loss_mode", C.c_int32), ("loss_body", C.c_int32),
                ("exact_mlp", C.c_int32), ("warmstart", C.c_int32), ("ws_W", PD), ("ws_alpha", C.c_double),
                ("grad_decay", C.c_double), ("n_recurrent", C.c_int32)]

WS_IN, WS_H, WS_OUT = 16, 64, 3
WS_PARAMS = WS_IN * WS_H + WS_H + WS_H * WS_H + WS_H + WS_H * WS_OUT + WS_OUT


INST_FIELDS = ("mass", "inertia", "anchor", "axis", "ref", "limit", "motor", "sph_off", "sph_rad", "sph_mu",
               "sph_e", "loss_point", "loss_target", "state0")


class Inst(C.Structure):
    _fields_ = [(k, PD) for k in INST_FIELDS]


class Grad(C.Structure):
    _fields_ = [(k, PD) for k in INST_FIELDS + ("W",)]


def _ip(a):
    return a.ctypes.data_as(PI)


def _dp(a):
    return a.ctypes.data_as(PD)


class _Keep:
    """Holds the numpy buffers referenced by a ctypes structure."""

    def __init__(self):
        self.refs = []

    def i32(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
        if a.size == 0:
            a = np.zeros(1, np.int32)
        self.refs.append(a)
        return _ip(a)

    def f64(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        if a.size == 0:
            a = np.zeros(1, np.float64)
        self.refs.append(a)
        return _dp(a)


def topo(m, keep, iters=None):
    t = Topo()
    t.nb, t.nj, t.ns, t.np = m.nb, m.nj, m.ns, m.np_
    t.joint_type = keep.i32(m.joint_type)
    t.joint_body = keep.i32(m.joint_body)
    t.joint_flags = keep.i32(m.joint_flags)
    t.sphere_body = keep.i32(m.sphere_body)
    t.pair_sphere = keep.i32(m.pair_sphere)
    t.n_layers = max(len(m.widths) - 1, 0)
    t.widths = keep.i32(m.widths if m.widths else [0])
    t.skip = m.skip
    t.features = m.features
    t.imu_body = m.imu_body
    t.clock_hz = m.clock_hz
    for k in range(3):
        t.gravity[k] = m.gravity[k]
    t.dt, t.ground_z, t.beta, t.gamma, t.slop = m.dt, m.ground_z, m.beta, m.gamma, m.slop
    t.iters = m.iters if iters is None else iters
    t.loss_kind, t.loss_mode, t.loss_body = m.loss_kind, m.loss_mode, m.loss_body
    t.exact_mlp = int(getattr(m, "exact_mlp", 0) or getattr(m, "ctrl_fp32", 0))
    ws = getattr(m, "ws_W", None)
    t.warmstart = int(bool(getattr(m, "warmstart", 0)) and ws is not None)
    t.ws_W = keep.f64(ws) if t.warmstart else None
    t.ws_alpha = float(getattr(m, "ws_alpha", 0.7))
    t.grad_decay = float(getattr(m, "grad_decay", 1.0))
    t.n_recurrent = int(getattr(m, "n_recurrent", 0))
    return t


def inst(m, i, keep, state0=None, overrides=None):
    s = Inst()
    for k in INST_FIELDS:
        a = getattr(m, k)[i]
        if k == "state0" and state0 is not None:
            a = state0
        if overrides and k in overrides:
            a = overrides[k]
        setattr(s, k, keep.f64(a))
    return s


def weights(m, keep, W=None):
    W = m.W if W is None else W
    if W is None or len(W) == 0:
        return keep.f64(np.zeros(1))
    return keep.f64(np.asarray(W, dtype=np.float64))


def n_slots(m):
    keep = _Keep()
    return lib().orc_num_slots(C.byref(topo(m, keep)))


def schedule(m):
    """Static row schedule: dict of per-slot kind, idx, sub, body_a, body_b, colour and the
    sweep order."""
    keep = _Keep()
    t = topo(m, keep)
    n = lib().orc_num_slots(C.byref(t))
    out = {k: np.zeros(max(n, 1), np.int32) for k in ("kind", "idx", "sub", "body_a", "body_b", "colour", "order")}
    r = lib().orc_schedule(C.byref(t), *[_ip(out[k]) for k in ("kind", "idx", "sub", "body_a", "body_b", "colour", "order")])
    assert r == n
    return {k: v[:n] for k, v in out.items()}


def rollout(m, i, horizon=None, W=None, log=False, iters=None, overrides=None, margins=False):
    """Roll instance ``i`` forward. Returns (states [T+1, nb, 18], loss, active, gap); with
    ``margins`` also the per-step bfloat16 tie margins [T]."""
    T = m.horizon if horizon is None else horizon
    keep = _Keep()
    t = topo(m, keep, iters)
    s = inst(m, i, keep, overrides=overrides)
    ns = lib().orc_num_slots(C.byref(t))
    states = np.zeros((T + 1, m.nb, 18))
    loss = C.c_double(0.0)
    active = np.zeros((T, max(ns, 1)), np.int8) if log else None
    gap = np.zeros((T, max(ns, 1))) if log else None
    marg = np.zeros(max(T, 1)) if margins else None
    r = lib().orc_rollout(C.byref(t), C.byref(s), weights(m, keep, W), T, _dp(states), C.byref(loss),
                          active.ctypes.data_as(C.POINTER(C.c_int8)) if log else None,
                          _dp(gap) if log else None, _dp(marg) if margins else None)
    if r != 0:
        raise ValueError("oracle rejected the model")
    out = (states, loss.value, active[:, :ns] if log else None, gap[:, :ns] if log else None)
    return out + (marg[:T],) if margins else out


def step(m, i, x, t=0, W=None, iters=None, margins=False):
    """One step from state ``x`` [nb, 18] at step index ``t``; returns (x_next, active, gap, lambda)
    and, with ``margins``, the step's bfloat16 tie margin."""
    keep = _Keep()
    tp = topo(m, keep, iters)
    s = inst(m, i, keep)
    ns = lib().orc_num_slots(C.byref(tp))
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1))
    xn = np.zeros_like(x)
    active = np.zeros(max(ns, 1), np.int8)
    gap = np.zeros(max(ns, 1))
    lam = np.zeros(max(ns, 1))
    marg = np.zeros(1)
    r = lib().orc_step(C.byref(tp), C.byref(s), weights(m, keep, W), t, _dp(x), _dp(xn),
                       active.ctypes.data_as(C.POINTER(C.c_int8)), _dp(gap), _dp(lam), _dp(marg))
    if r != 0:
        raise ValueError("oracle rejected the model")
    out = (xn.reshape(m.nb, 18), active[:ns], gap[:ns], lam[:ns])
    return out + (float(marg[0]),) if margins else out


def rollout_grad(m, i, horizon=None, W=None, iters=None, overrides=None):
    """Loss and gradient dict (same keys/shapes as the per-instance fields, plus ``W``)."""
    T = m.horizon if horizon is None else horizon
    keep = _Keep()
    t = topo(m, keep, iters)
    s = inst(m, i, keep, overrides=overrides)
    g = Grad()
    out = {}
    for k in INST_FIELDS:
        out[k] = np.zeros(getattr(m, k)[i].shape)
        setattr(g, k, keep.f64(out[k]) if out[k].size else None)
        out[k] = keep.refs[-1].reshape(out[k].shape) if out[k].size else out[k]
    nW = 0 if m.W is None else len(m.W)
    out["W"] = np.zeros(max(nW, 1))
    g.W = _dp(out["W"])
    loss = C.c_double(0.0)
    r = lib().orc_rollout_grad(C.byref(t), C.byref(s), weights(m, keep, W), T, C.byref(loss), C.byref(g))
    if r != 0:
        raise ValueError("oracle rejected the model")
    out["W"] = out["W"][:nW]
    return loss.value, out


def param_count(widths, skip=0):
    w = np.asarray(widths, np.int32)
    return lib().orc_param_count(len(widths) - 1, _ip(w), skip)


def bf16(x):
    return lib().orc_bf16(float(x))


def flops(m, i=0, horizon=None, W=None):
    """Algorithmic operations per step of instance ``i``: (forward, reverse, tape nodes)."""
    T = m.horizon if horizon is None else horizon
    keep = _Keep()
    t = topo(m, keep)
    s = inst(m, i, keep)
    out = np.zeros(3)
    r = lib().orc_flops(C.byref(t), C.byref(s), weights(m, keep, W), T, _dp(out))
    if r != 0:
        raise ValueError("oracle rejected the model")
    return tuple(out)


def step_log(m, i, x, t=0, W=None, iters=None, lam_prev=None, h_prev=None):
    """One step from state ``x`` with the full step record: dict with ``xn`` [nb, 18], ``active``,
    ``gap``, ``lam`` (final impulses), ``lam0`` (initial impulses), ``margin`` (bfloat16 tie
    margin), ``resid`` (RMS residual of the solve) and ``feats`` [groups, 16] (warm-start
    features of every group, see ``ws_groups``) and ``h`` (the controller's next recurrent
    state). ``lam_prev`` [n_slots]: the impulses the previous step ended with (default zeros);
    ``h_prev`` [n_recurrent]: the controller's recurrent state (default zeros)."""
    keep = _Keep()
    tp = topo(m, keep, iters)
    s = inst(m, i, keep)
    ns = lib().orc_num_slots(C.byref(tp))
    nc = lib().orc_ws_groups(C.byref(tp))
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1))
    xn = np.zeros_like(x)
    active = np.zeros(max(ns, 1), np.int8)
    gap, lam, lam0 = np.zeros(max(ns, 1)), np.zeros(max(ns, 1)), np.zeros(max(ns, 1))
    marg, resid = np.zeros(1), np.zeros(1)
    feats = np.zeros((max(nc, 1), WS_IN))
    H = int(getattr(m, "n_recurrent", 0))
    hn = np.zeros(max(H, 1))
    r = lib().orc_step_log(C.byref(tp), C.byref(s), weights(m, keep, W), t, _dp(x), _dp(xn),
                           active.ctypes.data_as(C.POINTER(C.c_int8)), _dp(gap), _dp(lam), _dp(marg), _dp(resid),
                           _dp(feats), _dp(lam0),
                           keep.f64(lam_prev) if lam_prev is not None else None,
                           keep.f64(h_prev) if h_prev is not None else None, _dp(hn))
    if r != 0:
        raise ValueError("oracle rejected the model")
    return dict(xn=xn.reshape(m.nb, 18), active=active[:ns], gap=gap[:ns], lam=lam[:ns], lam0=lam0[:ns],
                margin=float(marg[0]), resid=float(resid[0]), feats=feats[:nc], h=hn[:H])


def rollout_rec(m, i, horizon=None, W=None, iters=None):
    """Rollout of instance ``i`` with the controller's recurrent state of every step:
    (states [T+1, nb, 18], loss, h [T+1, n_recurrent]); h[0] = 0."""
    T = m.horizon if horizon is None else horizon
    keep = _Keep()
    t = topo(m, keep, iters)
    s = inst(m, i, keep)
    H = int(getattr(m, "n_recurrent", 0))
    states = np.zeros((T + 1, m.nb, 18))
    hs = np.zeros((T + 1, max(H, 1)))
    loss = C.c_double(0.0)
    r = lib().orc_rollout_rec(C.byref(t), C.byref(s), weights(m, keep, W), T, _dp(states), C.byref(loss), _dp(hs))
    if r != 0:
        raise ValueError("oracle rejected the model")
    return states, loss.value, hs[:, :H]


def rollout_resid(m, i, horizon=None, W=None, iters=None):
    """Rollout of instance ``i`` with the residual of every step's solve: (states, loss, resid [T])."""
    T = m.horizon if horizon is None else horizon
    keep = _Keep()
    t = topo(m, keep, iters)
    s = inst(m, i, keep)
    states = np.zeros((T + 1, m.nb, 18))
    resid = np.zeros(max(T, 1))
    loss = C.c_double(0.0)
    r = lib().orc_rollout_log(C.byref(t), C.byref(s), weights(m, keep, W), T, _dp(states), C.byref(loss), None, None,
                              None, _dp(resid))
    if r != 0:
        raise ValueError("oracle rejected the model")
    return states, loss.value, resid[:T]


def ws_loss_grad(Wws, rows, exact=False):
    """Mean squared error of the warm-start network over harvested rows [n, 19] and its gradient
    [WS_PARAMS] (bfloat16 storage points unless ``exact``)."""
    Wws = np.ascontiguousarray(np.asarray(Wws, np.float64).reshape(-1))
    rows = np.ascontiguousarray(np.asarray(rows, np.float64).reshape(-1, 19))
    assert Wws.size == WS_PARAMS
    loss = C.c_double(0.0)
    dW = np.zeros(WS_PARAMS)
    r = lib().orc_ws_loss_grad(_dp(Wws), _dp(rows), C.c_int64(rows.shape[0]), int(exact), C.byref(loss), _dp(dW))
    if r != 0:
        raise ValueError("oracle rejected the rows")
    return loss.value, dW


def ws_forward(Wws, feats, exact=False):
    """Warm-start network outputs [n, 3] for features [n, 16]."""
    Wws = np.ascontiguousarray(np.asarray(Wws, np.float64).reshape(-1))
    feats = np.ascontiguousarray(np.asarray(feats, np.float64).reshape(-1, WS_IN))
    y = np.zeros((feats.shape[0], WS_OUT))
    lib().orc_ws_forward(_dp(Wws), _dp(feats), C.c_int64(feats.shape[0]), int(exact), _dp(y))
    return y


WS_GROUND, WS_PAIR, WS_JOINT, WS_HINGE = 0, 1, 2, 3


def ws_groups(m):
    """Warm-start groups of a model, in the oracle's order: list of (type, (slot0, slot1, slot2)),
    derived from the slot schedule (joint linear rows, hinge angular rows + motor, contacts)."""
    sch = schedule(m)
    kind, idx, sub = sch["kind"], sch["idx"], sch["sub"]
    out = []
    for i in range(len(kind)):
        if kind[i] == 0 and sub[i] == 0:
            out.append((WS_JOINT, (i, i + 1, i + 2)))
        elif kind[i] == 1 and sub[i] == 0:
            mot = [k for k in range(len(kind)) if kind[k] == 3 and idx[k] == idx[i]]
            out.append((WS_HINGE, (i, i + 1, mot[-1] if mot else -1)))
        elif kind[i] == 4:
            out.append((WS_GROUND, (i, i + 1, i + 2)))
        elif kind[i] == 6:
            out.append((WS_PAIR, (i, i + 1, i + 2)))
    return out


# ----------------------------------------------------------------------------- camera
class Camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("f", C.c_double), ("plane", C.c_double), ("pos", C.c_double * 3),
                ("rot", C.c_double * 9)]


class Scene(C.Structure):
    _fields_ = [("n_obj", C.c_int32), ("body", PI), ("center", PD), ("half", PD), ("tex", PI), ("n_tex", C.c_int32),
                ("tex_h", C.c_int32), ("tex_w", C.c_int32), ("tex_data", PD), ("kind", PI)]


def _camera_scene(cs, keep, tex=None):
    cam = Camera()
    cam.W, cam.H, cam.f, cam.plane = int(cs.W), int(cs.H), float(cs.f), float(cs.plane)
    for k in range(3):
        cam.pos[k] = float(cs.cam_pos[k])
    for k in range(9):
        cam.rot[k] = float(np.asarray(cs.cam_rot).reshape(-1)[k])
    sc = Scene()
    sc.n_obj = len(cs.obj_body)
    sc.body, sc.center, sc.half, sc.tex = keep.i32(cs.obj_body), keep.f64(cs.obj_center), keep.f64(cs.obj_half), keep.i32(cs.obj_tex)
    t = np.asarray(cs.textures if tex is None else tex, np.float64)
    sc.n_tex, sc.tex_h, sc.tex_w = t.shape[0], t.shape[1], t.shape[2]
    sc.tex_data = keep.f64(t)
    kind = getattr(cs, "obj_kind", None)
    sc.kind = keep.i32(kind) if kind is not None else None
    return cam, sc


def render(cs, state, tex=None):
    """Frame [H, W, 3] of camera scene ``cs`` (see ``workloads.camera_scene``) for one state
    [nb, 18], and the box each pixel sees [H, W] (-1: none)."""
    keep = _Keep()
    cam, sc = _camera_scene(cs, keep, tex)
    state = np.ascontiguousarray(np.asarray(state, np.float64).reshape(-1))
    img = np.zeros((cs.H, cs.W, 3))
    hit = np.zeros((cs.H, cs.W), np.int32)
    r = lib().orc_render(C.byref(cam), C.byref(sc), state.size // 18, _dp(state), _dp(img), _ip(hit))
    if r != 0:
        raise ValueError("oracle rejected the camera or scene")
    return img, hit


def render_grad(cs, state, dimage, tex=None):
    """Gradient of sum(dimage * frame) w.r.t. the state [nb, 18] and the textures."""
    keep = _Keep()
    cam, sc = _camera_scene(cs, keep, tex)
    state = np.ascontiguousarray(np.asarray(state, np.float64).reshape(-1))
    dimage = np.ascontiguousarray(np.asarray(dimage, np.float64).reshape(-1))
    ds = np.zeros_like(state)
    t = np.asarray(cs.textures if tex is None else tex)
    dt = np.zeros(t.shape)
    r = lib().orc_render_grad(C.byref(cam), C.byref(sc), state.size // 18, _dp(state), _dp(dimage), _dp(ds), _dp(dt))
    if r != 0:
        raise ValueError("oracle rejected the camera or scene")
    return ds.reshape(-1, 18), dt
