"""Differentiable camera (section 3.4) through the C ABI against the FP64 oracle: frames of the
camera scene (the 3-link pendulum in front of a textured backdrop; boxes only, and mixed with a
sphere on the last link and a textured ground plane), the object each pixel sees, and the
reverse mode to the body poses and the texels; also at the full 288 x 96 size in the
4096-frame launch configuration the bench times, on sampled instances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import CameraRig  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_frames(cs, states):
    rig = CameraRig(cs)
    st = torch.tensor(np.asarray(states, np.float32), device="cuda")
    tex = torch.tensor(np.asarray(cs.textures, np.float32), device="cuda")
    img = torch.zeros(st.shape[0], cs.H, cs.W, 3, device="cuda")
    hit = torch.zeros(st.shape[0], cs.H, cs.W, dtype=torch.int32, device="cuda")
    rig.render(st, tex, img, hit)
    torch.cuda.synchronize()
    return rig, st, tex, img.cpu().numpy(), hit.cpu().numpy()


def compare(cs, states, inst, img, hit):
    """Hit sets equal except at silhouette pixels where fp32 and FP64 may pick different boxes
    (at most 0.2 % of the frame); where the same box is seen, colours within 1e-4 on at least
    99.9 % of the pixels (the rest: rays through a box edge, where the two precisions may enter
    through different faces of the same box)."""
    for i in inst:
        ref, rhit = O.render(cs, states[i])
        same = hit[i] == rhit
        assert same.mean() >= 0.998, (i, same.mean())
        err = np.abs(img[i] - ref).max(axis=-1)[same]
        assert (err <= 1e-4).mean() >= 0.999, (i, (err <= 1e-4).mean(), err.max())
    return True


@pytest.mark.parametrize("mixed", [False, True])
def test_frames_match_oracle(mixed):
    cs = WL.camera_scene(B=16, W=144, H=48, mixed=mixed)
    _, _, _, img, hit = gpu_frames(cs, cs.states)
    compare(cs, cs.states, range(16), img, hit)
    assert (hit >= 1).mean() > 0.005  # the pendulum is in view
    if mixed:
        assert (hit == 4).mean() > 1e-4 and (hit == 5).mean() > 0.05  # the sphere and the ground


@pytest.mark.parametrize("W,H,B,mixed", [(144, 48, 8, False), (288, 96, 4, False), (144, 48, 8, True),
                                         (288, 96, 4, True)])
def test_gradients_match_oracle(W, H, B, mixed):
    """Reverse mode of a random weighting of the frames: gradients w.r.t. the three link bodies'
    positions and rotation entries, and w.r.t. every texel, within 1e-3 (relative) of the
    oracle's, on instances whose hit sets agree everywhere; at 144 x 48 (the per-thread frame
    path) and at the full 288 x 96 (box frames staged per block)."""
    cs = WL.camera_scene(B=B, W=W, H=H, mixed=mixed)
    rig, st, tex, img, hit = gpu_frames(cs, cs.states)
    rng = np.random.default_rng(2)
    dimg = rng.normal(size=img.shape).astype(np.float32)
    ds = torch.zeros(st.shape, device="cuda")
    dt = torch.zeros(tex.shape, device="cuda")
    rig.render_backward(st, tex, torch.tensor(dimg, device="cuda"), ds, dt)
    torch.cuda.synchronize()
    ds, dt = ds.cpu().numpy(), dt.cpu().numpy()
    dt_ref = np.zeros(dt.shape)
    checked = 0
    for i in range(cs.states.shape[0]):
        rhit = O.render(cs, cs.states[i])[1]
        if not np.array_equal(hit[i], rhit):
            continue
        g, gt = O.render_grad(cs, cs.states[i], dimg[i])
        for b in range(3):
            if np.abs(g[b]).max() == 0.0:
                continue
            e = np.linalg.norm(ds[i, b] - g[b]) / np.linalg.norm(g[b])
            assert e <= 1e-3, (i, b, e)
        assert np.all(ds[i, :, 12:] == 0.0)
        checked += 1
    assert checked >= B // 2, checked
    # texel gradients summed over all instances (every instance's hits must agree for this sum)
    if all(np.array_equal(hit[i], O.render(cs, cs.states[i])[1]) for i in range(cs.states.shape[0])):
        for i in range(cs.states.shape[0]):
            dt_ref += O.render_grad(cs, cs.states[i], dimg[i])[1]
        e = np.linalg.norm(dt - dt_ref) / np.linalg.norm(dt_ref)
        assert e <= 1e-3, e


def test_full_size_batch_sampled():
    """4096 frames at 288 x 96 in one launch (the bench's configuration): sampled instances,
    including the last one, against the oracle."""
    cs = WL.camera_scene(B=4096, W=288, H=96)
    _, _, _, img, hit = gpu_frames(cs, cs.states)
    compare(cs, cs.states, [0, 1, 777, 2048, 4095], img, hit)


@pytest.mark.parametrize("mixed", [False, True])
def test_screen_rectangles_change_nothing(monkeypatch, mixed):
    """At 288 x 96 every block of pixels lies in one instance, and each object's screen rectangle
    lets the block's pixels skip the objects they cannot see. Without the rectangles
    (DP_CAMERA_NO_CULL) the frames and hit maps are the same bit for bit, and the gradients the
    same up to the order of the reverse pass's atomic sums."""
    cs = WL.camera_scene(B=32, W=288, H=96, mixed=mixed)
    outs = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("DP_CAMERA_NO_CULL", "1")
        rig, st, tex, img, hit = gpu_frames(cs, cs.states)
        dimg = np.random.default_rng(3).normal(size=img.shape).astype(np.float32)
        ds = torch.zeros(st.shape, device="cuda")
        dt = torch.zeros(tex.shape, device="cuda")
        rig.render_backward(st, tex, torch.tensor(dimg, device="cuda"), ds, dt)
        torch.cuda.synchronize()
        outs.append((img, hit, ds.cpu().numpy(), dt.cpu().numpy()))
    (ia, ha, sa, ta), (ib, hb, sb, tb) = outs
    assert np.array_equal(ia, ib) and np.array_equal(ha, hb)
    assert np.abs(sa - sb).max() <= 1e-5 * max(1.0, np.abs(sb).max())
    assert np.abs(ta - tb).max() <= 1e-5 * max(1.0, np.abs(tb).max())
