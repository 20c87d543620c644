"""C-ABI library: builds for sm_103a, loads, exports every symbol include/dp.h declares, and
rejects bad descriptors on the host (no GPU compute is called here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1611_01652_gb300 import binding, build, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.SYMBOLS) == set(names)


def test_enums_agree_with_header():
    src = open(HEADER).read()
    for name, val in (("DP_JOINT_HINGE", workloads.HINGE), ("DP_FLAG_MOTOR", workloads.FLAG_MOTOR),
                      ("DP_F_IMU", workloads.F_IMU), ("DP_LOSS_DISP", workloads.L_DISP), ("DP_MODE_MEAN", workloads.M_MEAN)):
        m = re.search(name + r"\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == val, name


def _desc(model):
    keep = []
    d = binding.BatchDesc()

    def i32(a):
        a = np.ascontiguousarray(np.asarray(a, np.int32).reshape(-1)) if np.size(a) else np.zeros(1, np.int32)
        keep.append(a)
        return a.ctypes.data_as(binding.PI)

    def f32(a):
        a = np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1)) if np.size(a) else np.zeros(1, np.float32)
        keep.append(a)
        return a.ctypes.data_as(binding.PF)

    d.n_instances, d.n_bodies, d.n_joints, d.n_spheres, d.n_pairs = model.B, model.nb, model.nj, model.ns, model.np_
    d.joint_type, d.joint_body, d.joint_flags = i32(model.joint_type), i32(model.joint_body), i32(model.joint_flags)
    d.sphere_body, d.pair_sphere = i32(model.sphere_body), i32(model.pair_sphere)
    for k in ("mass", "inertia", "anchor", "axis", "ref", "limit", "motor", "sph_off", "sph_rad", "sph_mu", "sph_e",
              "loss_point", "loss_target", "state0"):
        setattr(d, k, f32(getattr(model, k)))
    d.n_layers = max(len(model.widths) - 1, 0)
    for l, wv in enumerate(model.widths):
        d.widths[l] = wv
    d.features, d.imu_body, d.dt, d.iters, d.horizon = model.features, model.imu_body, model.dt, model.iters, model.horizon
    d.loss_kind, d.loss_mode, d.loss_body, d.beta, d.slop = model.loss_kind, model.loss_mode, model.loss_body, 0.2, 0.005
    d.gravity[2] = -9.81
    return d, keep


@pytest.mark.parametrize("mutate,needle", [
    (lambda d: setattr(d, "n_instances", 0), b"n_instances"),
    (lambda d: setattr(d, "horizon", 0), b"horizon"),
    (lambda d: setattr(d, "iters", 0), b"iters"),
    (lambda d: setattr(d, "n_bodies", 40), b"n_bodies"),
    (lambda d: setattr(d, "loss_body", 99), b"loss_body"),
    (lambda d: setattr(d, "n_layers", 9), b"n_layers"),
    (lambda d: setattr(d, "dt", -1.0), b"dt"),
])
def test_descriptor_validation_rejects_bad_input(mutate, needle):
    lib = binding.load()
    d, keep = _desc(workloads.quadruped(B=3, horizon=5))
    mutate(d)
    h = C.c_void_p()
    st = lib.dp_create_world(C.byref(d), None, C.byref(h))
    assert st == binding.DP_EINVAL
    assert not h.value
    assert needle in lib.dp_last_error()


def test_descriptor_validation_bad_topology():
    lib = binding.load()
    m = workloads.quadruped(B=2, horizon=5)
    m.joint_body = m.joint_body.copy()
    m.joint_body[3] = [2, 2]
    d, keep = _desc(m)
    h = C.c_void_p()
    assert lib.dp_create_world(C.byref(d), None, C.byref(h)) == binding.DP_EINVAL
    m = workloads.quadruped(B=2, horizon=5)
    m.mass = m.mass.copy()
    m.mass[1, 3] = 0.0
    d, keep = _desc(m)
    assert lib.dp_create_world(C.byref(d), None, C.byref(h)) == binding.DP_EINVAL
    assert b"mass" in lib.dp_last_error()


def test_null_world_calls_fail_cleanly():
    lib = binding.load()
    assert lib.dp_rollout(None, None, None, None, None) == binding.DP_EINVAL
    assert lib.dp_backward(None, None, None, None, None) == binding.DP_EINVAL
    assert lib.dp_num_slots(None) == -1
    lib.dp_free(None)


def test_build_flags_target_sm103a():
    assert "arch=compute_103a,code=sm_103a" in build.FLAGS


def test_recurrent_descriptor_validation():
    """n_recurrent out of range, or a network too narrow for the sensors plus the recurrent state,
    is rejected at world creation."""
    lib = binding.load()
    d, keep = _desc(workloads.quadruped(B=2, horizon=5))
    d.n_recurrent = -1
    h = C.c_void_p()
    assert lib.dp_create_world(C.byref(d), None, C.byref(h)) == binding.DP_EINVAL
    assert b"n_recurrent" in lib.dp_last_error()
    d.n_recurrent = 4  # 24 sensor inputs + 4 recurrent > widths[0] = 24
    st = lib.dp_create_world(C.byref(d), None, C.byref(h))
    assert st == binding.DP_EINVAL and not h.value
    assert b"recurrent" in lib.dp_last_error()


def test_new_world_calls_reject_null():
    lib = binding.load()
    assert lib.dp_set_params(None, None) == binding.DP_EINVAL
    assert lib.dp_set_recurrent(None, None) == binding.DP_EINVAL
    assert lib.dp_get_recurrent(None, None) == binding.DP_EINVAL


def _camera(n_obj=2, half=0.5):
    cam = binding.Camera()
    cam.width, cam.height, cam.focal, cam.plane = 8, 4, 4.0, 0.05
    for k, v in enumerate((1.0, 0.0, 0.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0)):
        cam.rotation[k] = v
    keep = [np.full(n_obj, -1, np.int32), np.zeros((n_obj, 3), np.float32), np.full((n_obj, 3), half, np.float32),
            np.zeros(n_obj, np.int32)]
    sc = binding.Scene()
    sc.n_obj = n_obj
    sc.body = keep[0].ctypes.data_as(binding.PI)
    sc.center = keep[1].ctypes.data_as(binding.PF)
    sc.half = keep[2].ctypes.data_as(binding.PF)
    sc.tex = keep[3].ctypes.data_as(binding.PI)
    sc.n_tex, sc.tex_h, sc.tex_w = 1, 2, 2
    return cam, sc, keep


@pytest.mark.parametrize("case,needle", [
    ("too_many", b"n_obj"), ("flat_box", b"half extents"), ("bad_texture", b"texture"), ("bad_camera", b"positive"),
])
def test_camera_validation_rejects_bad_scene(case, needle):
    """Malformed cameras and scenes are rejected on the host with a message, before any launch."""
    lib = binding.load()
    cam, sc, keep = _camera(n_obj=17 if case == "too_many" else 2, half=0.0 if case == "flat_box" else 0.5)
    if case == "bad_texture":
        keep[3][1] = 5
    if case == "bad_camera":
        cam.focal = 0.0
    st = lib.dp_render(C.byref(cam), C.byref(sc), 1, 1, None, None, None, None, None)
    assert st == binding.DP_EINVAL
    assert needle in lib.dp_camera_last_error()
    st = lib.dp_render_backward(C.byref(cam), C.byref(sc), 1, 1, None, None, None, None, None, None)
    assert st == binding.DP_EINVAL


def _struct_members(src, name):
    """Member names of the C struct typedef `name` in declaration order."""
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*" + name + r"\s*;", src, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*(.*)$", decl, flags=re.S)
        for part in m.group(1).split(","):
            names.append(re.sub(r"\[.*?\]", "", part).replace("*", "").strip())
    return names


def test_batch_descriptor_layout_agrees_with_header():
    """The binding's ctypes descriptor lists the header's dp_batch_desc members in the same order
    (the launch-configuration fields rows_global, dw_splits and one_warp included)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    assert _struct_members(src, "dp_batch_desc") == [f[0] for f in binding.BatchDesc._fields_]


def test_autotuner_space_covers_both_mappings():
    """The uneven batch's autotuner times one warp per group with every row, tape and split choice,
    and four warps per group (the compiled topologies' kernels keep the rows on chip and the whole
    tape) with each split count."""
    from paper_1611_01652_gb300 import batching

    cands = batching.CANDIDATES
    four = [c for c in cands if not c["one_warp"]]
    one = [c for c in cands if c["one_warp"]]
    assert len(one) == 8 and len(four) == 2
    assert all(not c["rows_global"] and c["ckpt_every"] == 0 for c in four)
    assert {c["dw_splits"] for c in four} == {64, 256}
