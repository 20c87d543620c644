"""Thin ctypes binding of libdphys (include/dp.h): argument marshalling only.

Every step of a rollout and of its reverse mode runs in the library's CUDA kernels; there is no
CPU fallback. Pointers are taken from torch tensors (device or host) or numpy arrays (host).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DP_OK, DP_EINVAL, DP_ENOMEM, DP_ECUDA, DP_ETIMEOUT, DP_ENAN, DP_ESTATE = range(7)
MAX_LAYERS = 6
PARAM_GRADS = ("mass", "inertia", "anchor", "limit", "motor", "sph_off", "sph_rad", "sph_mu", "sph_e", "loss_point",
               "loss_target")

PF = C.POINTER(C.c_float)
PI = C.POINTER(C.c_int32)


class BatchDesc(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("n_bodies", C.c_int32), ("n_joints", C.c_int32),
                ("n_spheres", C.c_int32), ("n_pairs", C.c_int32),
                ("joint_type", PI), ("joint_body", PI), ("joint_flags", PI), ("sphere_body", PI), ("pair_sphere", PI),
                ("mass", PF), ("inertia", PF), ("anchor", PF), ("axis", PF), ("ref", PF), ("limit", PF),
                ("motor", PF), ("sph_off", PF), ("sph_rad", PF), ("sph_mu", PF), ("sph_e", PF),
                ("loss_point", PF), ("loss_target", PF), ("state0", PF),
                ("n_layers", C.c_int32), ("widths", C.c_int32 * (MAX_LAYERS + 1)), ("skip", C.c_int32),
                ("features", C.c_int32), ("imu_body", C.c_int32), ("clock_hz", C.c_float),
                ("gravity", C.c_float * 3), ("dt", C.c_float), ("ground_z", C.c_float), ("beta", C.c_float),
                ("gamma", C.c_float), ("slop", C.c_float), ("iters", C.c_int32), ("horizon", C.c_int32),
                ("ckpt_every", C.c_int32), ("loss_kind", C.c_int32), ("loss_mode", C.c_int32),
                ("loss_body", C.c_int32), ("ctrl_fp32", C.c_int32), ("warmstart", C.c_int32),
                ("horizons", PI), ("rows_global", C.c_int32), ("dw_splits", C.c_int32), ("grad_decay", C.c_float),
                ("n_recurrent", C.c_int32), ("one_warp", C.c_int32)]

WS_PARAMS = 5443
WS_ROW = 19


class ParamGrads(C.Structure):
    _fields_ = [(k, PF) for k in PARAM_GRADS]


_lib = None
SYMBOLS = ("dp_create_world", "dp_free", "dp_num_params", "dp_num_slots", "dp_schedule", "dp_set_initial_state",
           "dp_set_state", "dp_get_state", "dp_step", "dp_rollout", "dp_backward", "dp_sync", "dp_last_error",
           "dp_ckpt_every", "dp_backward_noalloc", "dp_set_warmstart", "dp_harvest", "dp_set_residual",
           "dp_get_residual", "dp_ws_workspace_floats", "dp_ws_param_count", "dp_ws_loss_grad", "dp_ws_forward",
           "dp_ws_adam", "dp_set_impulses", "dp_get_impulses", "dp_set_recurrent", "dp_get_recurrent",
           "dp_set_params", "dp_render", "dp_render_backward", "dp_camera_last_error", "dp_instance_status",
           "dp_last_error_detail", "dp_fma_peak", "dp_controller_kind")
INST_NAN_STATE, INST_NAN_GRAD = 1, 2
CTRL_NONE, CTRL_SIMT, CTRL_TENSOR, CTRL_WIDE = 0, 1, 2, 3


def load(build=True):
    """Load libdphys.so (building it first if needed). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libdphys.so is missing: run paper_1611_01652_gb300.build.build()")
    lib = C.CDLL(path)
    lib.dp_create_world.argtypes = [C.POINTER(BatchDesc), C.c_void_p, C.POINTER(C.c_void_p)]
    lib.dp_free.argtypes = [C.c_void_p]
    lib.dp_free.restype = None
    lib.dp_num_params.argtypes = [C.c_void_p]
    lib.dp_num_params.restype = C.c_int64
    lib.dp_num_slots.argtypes = [C.c_void_p]
    lib.dp_ckpt_every.argtypes = [C.c_void_p]
    lib.dp_controller_kind.argtypes = [C.c_void_p]
    lib.dp_schedule.argtypes = [C.c_void_p] + [PI] * 7
    lib.dp_set_initial_state.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    lib.dp_get_state.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_step.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
    lib.dp_rollout.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dp_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(ParamGrads)]
    lib.dp_backward_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dp_sync.argtypes = [C.c_void_p]
    lib.dp_instance_status.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_fma_peak.argtypes = [C.c_int64, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]
    lib.dp_last_error_detail.argtypes = [C.c_void_p, C.c_char_p, C.c_size_t]
    lib.dp_last_error.restype = C.c_char_p
    lib.dp_set_warmstart.argtypes = [C.c_void_p, C.c_void_p, C.c_float]
    lib.dp_set_impulses.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_get_impulses.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_set_recurrent.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_set_params.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_render.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p]
    lib.dp_render_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dp_camera_last_error.restype = C.c_char_p
    lib.dp_get_recurrent.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_harvest.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
    lib.dp_set_residual.argtypes = [C.c_void_p, C.c_int32]
    lib.dp_get_residual.argtypes = [C.c_void_p, C.c_void_p]
    lib.dp_ws_workspace_floats.argtypes = [C.c_int64]
    lib.dp_ws_workspace_floats.restype = C.c_int64
    lib.dp_ws_param_count.restype = C.c_int32
    lib.dp_ws_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dp_ws_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dp_ws_adam.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_float,
                               C.c_float, C.c_float, C.c_float, C.c_void_p]
    _lib = lib
    return lib


class DPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dp status %d: %s" % (status, msg))
        self.status = status


def _check(status):
    if status != DP_OK:
        raise DPError(status, _lib.dp_last_error().decode())


def torch_float32():
    import torch

    return torch.float32


def ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


class World:
    """A batch of robots with one topology living on the current CUDA device.

    ``model`` is any object with the attributes of ``workloads.Model``. All calls are ordered on
    ``stream`` (a torch.cuda.Stream, default: the current stream at creation). ``rows_global``,
    ``dw_splits`` and ``one_warp`` are launch-configuration choices (the descriptor fields of the
    same names), which the results do not depend on beyond summation order.
    """

    def __init__(self, model, stream=None, ckpt_every=None, horizon=None, iters=None, warmstart=False,
                 rows_global=False, dw_splits=0, one_warp=False):
        import torch

        lib = load()
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.B, self.nb = int(model.B), int(model.nb)
        self._keep = []
        d = BatchDesc()

        def i32(a):
            a = np.ascontiguousarray(np.asarray(a, np.int32).reshape(-1))
            if a.size == 0:
                a = np.zeros(1, np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(PI)

        def f32(a):
            a = np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1))
            if a.size == 0:
                a = np.zeros(1, np.float32)
            self._keep.append(a)
            return a.ctypes.data_as(PF)

        d.n_instances = self.B
        d.n_bodies, d.n_joints, d.n_spheres, d.n_pairs = model.nb, model.nj, model.ns, model.np_
        d.joint_type, d.joint_body, d.joint_flags = i32(model.joint_type), i32(model.joint_body), i32(model.joint_flags)
        d.sphere_body, d.pair_sphere = i32(model.sphere_body), i32(model.pair_sphere)
        for k in ("mass", "inertia", "anchor", "axis", "ref", "limit", "motor", "sph_off", "sph_rad", "sph_mu", "sph_e",
                  "loss_point", "loss_target", "state0"):
            setattr(d, k, f32(getattr(model, k)))
        widths = list(model.widths) if model.widths else []
        d.n_layers = max(len(widths) - 1, 0)
        for l, wv in enumerate(widths):
            d.widths[l] = wv
        d.skip, d.features, d.imu_body, d.clock_hz = model.skip, model.features, model.imu_body, model.clock_hz
        for k in range(3):
            d.gravity[k] = model.gravity[k]
        d.dt, d.ground_z, d.beta, d.gamma, d.slop = model.dt, model.ground_z, model.beta, model.gamma, model.slop
        d.iters = model.iters if iters is None else iters
        d.horizon = model.horizon if horizon is None else horizon
        d.ckpt_every = model.ckpt_every if ckpt_every is None else ckpt_every
        d.loss_kind, d.loss_mode, d.loss_body = model.loss_kind, model.loss_mode, model.loss_body
        d.ctrl_fp32 = int(getattr(model, "ctrl_fp32", 0))
        d.warmstart = int(bool(warmstart))
        hz = getattr(model, "horizons", None)
        d.horizons = i32(np.minimum(hz, d.horizon)) if hz is not None else None
        d.rows_global = int(bool(rows_global))
        d.dw_splits = int(dw_splits)
        d.one_warp = int(bool(one_warp))
        d.grad_decay = float(getattr(model, "grad_decay", 1.0))
        d.n_recurrent = int(getattr(model, "n_recurrent", 0))
        self.n_recurrent = d.n_recurrent
        self.horizon = d.horizon
        self.n_motors = int(sum(1 for f in np.asarray(model.joint_flags).reshape(-1) if f & 2))
        h = C.c_void_p()
        _check(lib.dp_create_world(C.byref(d), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self._keep = []
        self.n_params = int(lib.dp_num_params(h))
        self.n_slots = int(lib.dp_num_slots(h))
        self.ckpt_every = int(lib.dp_ckpt_every(h))
        # DP_CTRL_*: none, SIMT in the step, tensor cores in the step, wide batched products
        self.controller_kind = int(lib.dp_controller_kind(h))

    # -- lifetime
    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.dp_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # -- calls (same names as the C ABI)
    def schedule(self):
        n = self.n_slots
        out = {k: np.zeros(max(n, 1), np.int32) for k in ("kind", "idx", "sub", "body_a", "body_b", "colour", "order")}
        _check(_lib.dp_schedule(self._h, *[out[k].ctypes.data_as(PI) for k in
                                          ("kind", "idx", "sub", "body_a", "body_b", "colour", "order")]))
        return {k: v[:n] for k, v in out.items()}

    def set_initial_state(self, state):
        _check(_lib.dp_set_initial_state(self._h, ptr(state)))

    def set_state(self, state, t=0):
        _check(_lib.dp_set_state(self._h, ptr(state), int(t)))

    def get_state(self, out):
        _check(_lib.dp_get_state(self._h, ptr(out)))
        return out

    def step(self, n_steps, W=None, active=None):
        _check(_lib.dp_step(self._h, int(n_steps), ptr(W), ptr(active)))

    def rollout(self, W, loss, traj=None, active=None):
        _check(_lib.dp_rollout(self._h, ptr(W), ptr(loss), ptr(traj), ptr(active)))
        return loss

    def backward(self, dloss, dW=None, dstate0=None, dparams=None):
        pg = None
        if dparams:
            pg = ParamGrads()
            for k in PARAM_GRADS:
                v = dparams.get(k)
                setattr(pg, k, C.cast(ptr(v), PF) if v is not None else None)
        _check(_lib.dp_backward(self._h, ptr(dloss), ptr(dW), ptr(dstate0), C.byref(pg) if pg is not None else None))

    def set_params(self, **groups):
        """Replace per-instance parameter groups in place (``mass=``, ``sph_e=``, ... arrays of the
        model's shapes, host or device); the next backward needs a new rollout."""
        pg = ParamGrads()
        keep = []
        for k in PARAM_GRADS:
            v = groups.pop(k, None)
            if isinstance(v, np.ndarray):
                v = np.ascontiguousarray(v, np.float32)
                keep.append(v)
            elif v is not None and v.dtype != torch_float32():
                raise TypeError("%s must be float32" % k)
            setattr(pg, k, C.cast(ptr(v), PF) if v is not None else None)
        if groups:
            raise ValueError("unknown parameter groups: %s" % sorted(groups))
        _check(_lib.dp_set_params(self._h, C.byref(pg)))

    def backward_noalloc(self, dloss, dW):
        """dL/dW through the last rollout without any device allocation (static scratch)."""
        _check(_lib.dp_backward_noalloc(self._h, ptr(dloss), ptr(dW)))

    def sync(self):
        _check(_lib.dp_sync(self._h))

    def instance_status(self, out):
        """Per-instance status flags into ``out`` ([B] int32, host or device): bit INST_NAN_STATE
        (non-finite state or loss), bit INST_NAN_GRAD (non-finite gradient in the last backward)."""
        _check(_lib.dp_instance_status(self._h, ptr(out)))
        return out

    def error_detail(self):
        """(status, one-line report of the flagged instances and the last error)."""
        buf = C.create_string_buffer(1024)
        st = _lib.dp_last_error_detail(self._h, buf, len(buf))
        return st, buf.value.decode()

    def set_warmstart(self, W, alpha=0.7):
        """Enable the learned warm start with network parameters W [WS_PARAMS] and weight alpha
        of the previous step's impulses (W = None: cold start)."""
        _check(_lib.dp_set_warmstart(self._h, ptr(W), float(alpha)))

    def set_impulses(self, lam):
        _check(_lib.dp_set_impulses(self._h, ptr(lam)))

    def get_impulses(self, out):
        _check(_lib.dp_get_impulses(self._h, ptr(out)))

    def set_recurrent(self, h):
        """The controller's recurrent state [B, n_recurrent] the next step starts from."""
        _check(_lib.dp_set_recurrent(self._h, ptr(h)))

    def get_recurrent(self, out):
        """Reads the controller's current recurrent state into ``out`` [B, n_recurrent]."""
        _check(_lib.dp_get_recurrent(self._h, ptr(out)))
        return out

    def harvest(self, W, rows, u_noise=None):
        """Rollout harvesting (features, ideal network output) rows into ``rows`` [max_rows, 19]
        (device); returns the number of rows written."""
        n = C.c_int64(0)
        _check(_lib.dp_harvest(self._h, ptr(W), ptr(u_noise), ptr(rows), int(rows.shape[0]), C.byref(n)))
        return int(n.value)

    def set_residual(self, on=True):
        _check(_lib.dp_set_residual(self._h, int(bool(on))))

    def get_residual(self, out):
        _check(_lib.dp_get_residual(self._h, ptr(out)))
        return out


# -- warm-start network training (free functions of the C ABI)
def ws_workspace(n, device="cuda"):
    import torch

    load()
    return torch.empty(int(_lib.dp_ws_workspace_floats(int(n))), device=device, dtype=torch.float32)


def ws_loss_grad(W, rows, loss, dW, work, stream=None):
    load()
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.dp_ws_loss_grad(ptr(W), ptr(rows), int(rows.shape[0]), ptr(loss), ptr(dW), ptr(work), s))


def ws_forward(W, feats, y, work, stream=None):
    load()
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.dp_ws_forward(ptr(W), ptr(feats), int(feats.shape[0]), ptr(y), ptr(work), s))


def ws_adam(W, dW, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    load()
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.dp_ws_adam(ptr(W), ptr(dW), ptr(m), ptr(v), int(W.numel()), int(step), float(lr), float(beta1),
                           float(beta2), float(eps), s))


def fma_peak(iters=4096, repeats=5):
    """Measured FP32 FMA throughput of the current device (FLOP/s): the best of ``repeats`` timed
    launches of the library's FMA kernel (CUDA events on the current stream, after one warm-up)."""
    import torch

    load()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sink = torch.empty(8 * props.multi_processor_count * 256, device="cuda")
    st = torch.cuda.current_stream()
    fl = C.c_int64(0)
    best = 0.0
    for r in range(repeats + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(_lib.dp_fma_peak(int(iters), ptr(sink), C.byref(fl), C.c_void_p(st.cuda_stream)))
        e1.record(st)
        e1.synchronize()
        if r > 0:
            best = max(best, fl.value / (e0.elapsed_time(e1) * 1e-3))
    return best


def make_rollout_function():
    """torch.autograd.Function: loss[B] = rollout(W, state0) through a World; backward returns
    dL/dW and dL/dstate0 from the library's reverse-mode kernels."""
    import torch

    class Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, W, state0, world):
            # the library reads float32: inputs of another dtype are converted (gradients are
            # returned in the inputs' dtypes)
            world.set_initial_state(state0.detach().to(torch.float32).contiguous())
            loss = torch.empty(world.B, device=state0.device, dtype=torch.float32)
            world.rollout(W.detach().to(torch.float32).contiguous() if W is not None else None, loss)
            ctx.world = world
            ctx.dtypes = (W.dtype if W is not None else None, state0.dtype)
            return loss

        @staticmethod
        def backward(ctx, gl):
            w = ctx.world
            dW = torch.empty(w.n_params, device=gl.device, dtype=torch.float32) if w.n_params else None
            ds = torch.empty(w.B, w.nb, 18, device=gl.device, dtype=torch.float32)
            w.backward(gl.contiguous().float(), dW, ds)
            tw, ts = ctx.dtypes
            return (dW.to(tw) if dW is not None else None), ds.to(ts), None

    return Rollout


# ----------------------------------------------------------------------------- camera
class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("focal", C.c_float), ("plane", C.c_float),
                ("position", C.c_float * 3), ("rotation", C.c_float * 9)]


class Scene(C.Structure):
    _fields_ = [("n_obj", C.c_int32), ("body", PI), ("center", PF), ("half", PF), ("tex", PI),
                ("n_tex", C.c_int32), ("tex_h", C.c_int32), ("tex_w", C.c_int32), ("kind", PI)]


class CameraRig:
    """The camera and scene of a ``workloads.CameraScene`` as the library's structures (host
    arrays kept alive here); ``textures`` is a device tensor the caller provides to each call."""

    def __init__(self, cs):
        load()
        self.cam = Camera()
        self.cam.width, self.cam.height, self.cam.focal, self.cam.plane = int(cs.W), int(cs.H), float(cs.f), float(cs.plane)
        for k in range(3):
            self.cam.position[k] = float(cs.cam_pos[k])
        for k in range(9):
            self.cam.rotation[k] = float(np.asarray(cs.cam_rot).reshape(-1)[k])
        self._keep = [np.ascontiguousarray(np.asarray(cs.obj_body, np.int32)),
                      np.ascontiguousarray(np.asarray(cs.obj_center, np.float32)),
                      np.ascontiguousarray(np.asarray(cs.obj_half, np.float32)),
                      np.ascontiguousarray(np.asarray(cs.obj_tex, np.int32)),
                      np.ascontiguousarray(np.asarray(getattr(cs, "obj_kind", np.zeros(len(cs.obj_body))), np.int32))]
        self.scene = Scene()
        self.scene.n_obj = len(self._keep[0])
        self.scene.body = self._keep[0].ctypes.data_as(PI)
        self.scene.center = self._keep[1].ctypes.data_as(PF)
        self.scene.half = self._keep[2].ctypes.data_as(PF)
        self.scene.tex = self._keep[3].ctypes.data_as(PI)
        self.scene.kind = self._keep[4].ctypes.data_as(PI)
        t = np.asarray(cs.textures)
        self.scene.n_tex, self.scene.tex_h, self.scene.tex_w = t.shape[0], t.shape[1], t.shape[2]
        self.nb = int(cs.nb)

    def _check(self, r):
        if r != 0:
            raise RuntimeError("camera call failed (status %d): %s" % (r, _lib.dp_camera_last_error().decode()))

    def render(self, state, textures, image, hit=None, stream=None):
        """Frames image [B, H, W, 3] of states [B, nb, 18] (device tensors)."""
        s = C.c_void_p(stream.cuda_stream) if stream is not None else None
        self._check(_lib.dp_render(C.byref(self.cam), C.byref(self.scene), int(state.shape[0]), self.nb, ptr(state),
                                   ptr(textures), ptr(image), ptr(hit), s))

    def render_backward(self, state, textures, dimage, dstate, dtextures=None, stream=None):
        """dstate [B, nb, 18] (and dtextures) of sum(dimage * image)."""
        s = C.c_void_p(stream.cuda_stream) if stream is not None else None
        self._check(_lib.dp_render_backward(C.byref(self.cam), C.byref(self.scene), int(state.shape[0]), self.nb,
                                            ptr(state), ptr(textures), ptr(dimage), ptr(dstate), ptr(dtextures), s))
