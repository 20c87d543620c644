"""Pins of the oracle's differentiable camera (section 3.4: pinhole rays through the pixel centres,
nearest hit in front of the projection plane, bilinear texture interpolation) against facts that
do not come from its own formulas: the pinhole geometry of a fronto-parallel face worked out
here, a linear texture (which bilinear interpolation reproduces exactly), the visibility rules,
and central differences of its forward pass (no GPU)."""
import numpy as np

import oracle as O
from paper_1611_01652_gb300.workloads import CameraScene

ROT_Y = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])  # look along +y, image down = -z


def scene(boxes, W=40, H=16, f=20.0, plane=0.05, tex=None, th=8, tw=8, kinds=None):
    """boxes: list of (body, centre, half, tex index); camera at the origin looking along +y;
    kinds: per object 0 (box) or 1 (sphere of radius half[0])."""
    cs = CameraScene()
    cs.W, cs.H, cs.f, cs.plane = W, H, f, plane
    cs.cam_pos = np.zeros(3)
    cs.cam_rot = ROT_Y
    cs.obj_body = np.array([b[0] for b in boxes], np.int32)
    cs.obj_center = np.array([b[1] for b in boxes], np.float64)
    cs.obj_half = np.array([b[2] for b in boxes], np.float64)
    cs.obj_tex = np.array([b[3] for b in boxes], np.int32)
    if tex is None:
        tex = np.random.default_rng(0).uniform(0, 1, size=(max(b[3] for b in boxes) + 1, th, tw, 3))
    cs.textures = tex
    if kinds is not None:
        cs.obj_kind = np.array(kinds, np.int32)
    return cs


def linear_texture(th, tw, coef):
    """Texel (r, c, ch) = a u_c + b v_r + c0 at the texel centres u_c = (c + 1/2)/tw, v_r = (r + 1/2)/th."""
    u = (np.arange(tw) + 0.5) / tw
    v = (np.arange(th) + 0.5) / th
    out = np.zeros((1, th, tw, 3))
    for ch, (a, b, c0) in enumerate(coef):
        out[0, :, :, ch] = a * u[None, :] + b * v[:, None] + c0
    return out


def test_fronto_parallel_face_with_linear_texture():
    """A world box whose -y face (x in [-hx, hx], z in [-hz, hz]) sits at distance D fills part of
    the view. The pixel (i, j) ray meets y = D at x = D ((j + 1/2) - W/2)/f, z = -D ((i + 1/2) -
    H/2)/f; the face's coordinates are u = (z / hz + 1)/2, v = (x / hx + 1)/2 (axis k = y, then z,
    then x); a texture linear in (u, v) comes back exactly wherever the sample is inside the
    texel-centre grid."""
    W, H, f, D = 40, 16, 20.0, 2.0
    hx, hy, hz = 1.5, 0.1, 0.6
    th, tw = 8, 8
    coef = [(0.3, 0.5, 0.1), (-0.2, 0.4, 0.5), (0.7, -0.1, 0.2)]
    cs = scene([(-1, [0.0, D + hy, 0.0], [hx, hy, hz], 0)], W, H, f, tex=linear_texture(th, tw, coef), th=th, tw=tw)
    img, hit = O.render(cs, np.zeros((0, 18)))
    checked = 0
    for i in range(H):
        for j in range(W):
            x = D * ((j + 0.5) - W / 2) / f
            z = -D * ((i + 0.5) - H / 2) / f
            inside = abs(x) <= hx and abs(z) <= hz
            assert hit[i, j] == (0 if inside else -1), (i, j)
            if not inside:
                assert np.all(img[i, j] == 0.0)
                continue
            u, v = (z / hz + 1) / 2, (x / hx + 1) / 2
            if not (0.5 / tw <= u <= 1 - 0.5 / tw and 0.5 / th <= v <= 1 - 0.5 / th):
                continue
            for ch, (a, b, c0) in enumerate(coef):
                assert abs(img[i, j, ch] - (a * u + b * v + c0)) <= 1e-12, (i, j, ch)
            checked += 1
    assert checked >= 100


def test_nearest_hit_in_front_of_the_projection_plane():
    """Along the optical axis: of two boxes the nearer is seen; a box between the camera and the
    projection plane, or behind the camera, is not seen."""
    near = (-1, [0.0, 1.0, 0.0], [0.3, 0.05, 0.3], 0)
    far = (-1, [0.0, 2.0, 0.0], [2.0, 0.05, 2.0], 1)
    inside_plane = (-1, [0.0, 0.02, 0.0], [0.5, 0.01, 0.5], 2)  # y in [0.01, 0.03] < plane 0.05
    behind = (-1, [0.0, -1.0, 0.0], [5.0, 0.05, 5.0], 3)
    cs = scene([far, behind, inside_plane, near])
    _, hit = O.render(cs, np.zeros((0, 18)))
    assert hit[8, 20] == 3  # the near box, index 3 in the list
    assert hit[0, 0] == 0  # beyond the near box's silhouette: the far backdrop
    assert not np.any(hit == 1) and not np.any(hit == 2)


def test_gradients_match_central_differences():
    """A body-carried box fills the view (no silhouette in the frame): the gradient of a random
    weighting of the frame with respect to the body's position and rotation entries and to the
    texels equals central differences of the forward pass."""
    rng = np.random.default_rng(1)
    th = tw = 6
    cs = scene([(0, [0.0, 0.0, 0.0], [4.0, 0.2, 3.0], 0)], W=24, H=10, f=10.0, th=th, tw=tw)
    ang = 0.2
    Rz = np.array([[np.cos(ang), -np.sin(ang), 0.0], [np.sin(ang), np.cos(ang), 0.0], [0.0, 0.0, 1.0]])
    x = np.zeros((1, 18))
    x[0, 0:3] = [0.1, 2.0, -0.05]
    x[0, 3:12] = Rz.reshape(-1)
    img, hit = O.render(cs, x)
    assert np.all(hit == 0)
    wgt = rng.normal(size=img.shape)
    ds, dt = O.render_grad(cs, x, wgt)

    def f(xx=None, tt=None):
        return float(np.sum(wgt * O.render(cs, x if xx is None else xx, tex=tt)[0]))

    for k in list(range(12)):
        eps = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[0, k] += eps
        xm[0, k] -= eps
        fd = (f(xp) - f(xm)) / (2 * eps)
        assert abs(fd - ds[0, k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, ds[0, k])
    assert np.all(ds[0, 12:] == 0.0)
    for idx in [(0, 2, 3, 0), (0, 0, 0, 1), (0, 5, 1, 2), (0, 3, 3, 1)]:
        eps = 1e-6
        tp, tm = cs.textures.copy(), cs.textures.copy()
        tp[idx] += eps
        tm[idx] -= eps
        fd = (f(tt=tp) - f(tt=tm)) / (2 * eps)
        assert abs(fd - dt[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, dt[idx])


def test_sphere_with_linear_texture():
    """A world sphere of radius r centred at (0, D, 0): the pixel (i, j) ray meets it where
    |t d - c| = r (near root), seen from outside; the hit direction p (from the centre) gives
    u = atan2(p_y, p_x) / (2 pi) + 1/2, v = acos(p_z / r) / pi, and a texture linear in (u, v)
    comes back exactly inside the texel-centre grid; rays that miss are black."""
    W, H, f, D, r = 40, 16, 20.0, 3.0, 1.0
    th, tw = 8, 8
    coef = [(0.3, 0.5, 0.1), (-0.2, 0.4, 0.5), (0.7, -0.1, 0.2)]
    cs = scene([(-1, [0.0, D, 0.0], [r, r, r], 0)], W, H, f, tex=linear_texture(th, tw, coef), th=th, tw=tw, kinds=[1])
    img, hit = O.render(cs, np.zeros((0, 18)))
    checked = 0
    for i in range(H):
        for j in range(W):
            d = np.array([((j + 0.5) - W / 2) / f, 1.0, -((i + 0.5) - H / 2) / f]) * cs.plane
            c = np.array([0.0, D, 0.0])
            a, b, cc = d @ d, d @ (-c), c @ c - r * r
            disc = b * b - a * cc
            if disc < 0:
                assert hit[i, j] == -1 and np.all(img[i, j] == 0.0), (i, j)
                continue
            assert hit[i, j] == 0, (i, j)
            p = ((-b - np.sqrt(disc)) / a) * d - c
            u = np.arctan2(p[1], p[0]) / (2 * np.pi) + 0.5
            v = np.arccos(np.clip(p[2] / r, -1, 1)) / np.pi
            if not (0.5 / tw <= u <= 1 - 0.5 / tw and 0.5 / th <= v <= 1 - 0.5 / th):
                continue
            for ch, (ca, cb, c0) in enumerate(coef):
                assert abs(img[i, j, ch] - (ca * u + cb * v + c0)) <= 1e-12, (i, j, ch)
            checked += 1
    assert checked >= 50


def test_sphere_occludes_box_and_gradients_match_central_differences():
    """A body-carried sphere in front of a backdrop box is seen where it covers the backdrop; a
    large sphere filling the frame (no silhouette) has the gradients of a random frame weighting
    w.r.t. its body's position and rotation entries and its texels equal central differences."""
    back = (-1, [0.0, 6.0, 0.0], [20.0, 0.1, 20.0], 0)
    ball = (0, [0.0, 0.0, 0.0], [0.5, 0.5, 0.5], 1)
    cs = scene([back, ball], kinds=[0, 1])
    x = np.zeros((1, 18))
    x[0, 0:3] = [0.0, 3.0, 0.0]
    x[0, 3:12] = np.eye(3).reshape(-1)
    _, hit = O.render(cs, x)
    assert hit[8, 20] == 1 and hit[0, 0] == 0
    rng = np.random.default_rng(3)
    cs = scene([(0, [0.0, 0.0, 0.0], [2.5, 2.5, 2.5], 0)], W=24, H=10, f=10.0, th=6, tw=6, kinds=[1])
    ang = 0.3
    R = np.array([[np.cos(ang), -np.sin(ang), 0.0], [np.sin(ang), np.cos(ang), 0.0], [0.0, 0.0, 1.0]])
    x[0, 0:3] = [0.05, 3.0, -0.1]
    x[0, 3:12] = R.reshape(-1)
    img, hit = O.render(cs, x)
    assert np.all(hit == 0)
    wgt = rng.normal(size=img.shape)
    ds, dt = O.render_grad(cs, x, wgt)

    def f(xx=None, tt=None):
        return float(np.sum(wgt * O.render(cs, x if xx is None else xx, tex=tt)[0]))

    for k in range(12):
        eps = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[0, k] += eps
        xm[0, k] -= eps
        fd = (f(xp) - f(xm)) / (2 * eps)
        assert abs(fd - ds[0, k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, ds[0, k])
    for idx in [(0, 2, 3, 0), (0, 4, 1, 2)]:
        eps = 1e-6
        tp, tm = cs.textures.copy(), cs.textures.copy()
        tp[idx] += eps
        tm[idx] -= eps
        fd = (f(tt=tp) - f(tt=tm)) / (2 * eps)
        assert abs(fd - dt[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, dt[idx])


def test_ground_plane_with_linear_texture_and_period():
    """A world plane z = -Z0 (kind 2: the plane z = 0 of a frame centred at (0, 0, -Z0)). The pixel
    (i, j) ray of the camera at the origin looking along +y meets it, for rows below the centre
    (i + 1/2 > H/2), at x = Z0 (j + 1/2 - W/2) / (i + 1/2 - H/2), y = Z0 f / (i + 1/2 - H/2), if
    that is beyond the projection plane (y >= P). The texture repeats with periods 2 h0, 2 h1:
    u = frac(x / (2 h0) + 1/2), v = frac(y / (2 h1) + 1/2); a texture linear in (u, v) comes back
    exactly inside the texel-centre grid. Moving the plane by one period along x leaves the frame
    unchanged; by half a period it does not."""
    W, H, f, Z0, P = 40, 20, 20.0, 1.0, 0.05
    h0, h1 = 0.7, 1.3
    th, tw = 8, 8
    coef = [(0.3, 0.5, 0.1), (-0.2, 0.4, 0.5), (0.7, -0.1, 0.2)]
    tex = linear_texture(th, tw, coef)

    def frame(x0):
        cs = scene([(-1, [x0, 0.0, -Z0], [h0, h1, 1.0], 0)], W, H, f, plane=P, tex=tex, th=th, tw=tw, kinds=[2])
        return O.render(cs, np.zeros((0, 18)))

    img, hit = frame(0.0)
    checked = 0
    for i in range(H):
        for j in range(W):
            di = (i + 0.5) - H / 2
            if di <= 0 or Z0 * f / di < P:
                assert hit[i, j] == -1 or di > 0
                continue
            assert hit[i, j] == 0, (i, j)
            x, y = Z0 * ((j + 0.5) - W / 2) / di, Z0 * f / di
            u = (x / (2 * h0) + 0.5) % 1.0
            v = (y / (2 * h1) + 0.5) % 1.0
            if not (0.5 / tw <= u <= 1 - 0.5 / tw and 0.5 / th <= v <= 1 - 0.5 / th):
                continue
            for ch, (a, b, c0) in enumerate(coef):
                assert abs(img[i, j, ch] - (a * u + b * v + c0)) <= 1e-12, (i, j, ch)
            checked += 1
    assert checked >= 40
    assert (hit[: H // 2] == -1).all()  # above the horizon nothing is seen
    img2, _ = frame(2 * h0)
    assert np.abs(img2 - img).max() <= 1e-9
    img3, _ = frame(h0)
    assert np.abs(img3 - img).max() > 1e-2


def test_body_carried_plane_gradients_match_central_differences():
    """A plane carried by a tilted body fills the lower half of the frame: the gradient of a
    random weighting of the frame with respect to the body's position and rotation entries and
    to the texels equals central differences of the forward pass."""
    rng = np.random.default_rng(4)
    W, H, f = 24, 12, 12.0
    cs = scene([(0, [0.0, 0.0, 0.0], [0.9, 1.1, 1.0], 0)], W, H, f, th=6, tw=6, kinds=[2])
    a = 0.15
    R = np.array([[1.0, 0.0, 0.0], [0.0, np.cos(a), -np.sin(a)], [0.0, np.sin(a), np.cos(a)]])
    x = np.zeros((1, 18))
    x[0, 0:3] = [0.1, 0.0, -1.0]
    x[0, 3:12] = R.reshape(-1)
    dimg = rng.normal(size=(H, W, 3))
    ds, dt = O.render_grad(cs, x, dimg)

    def fval(xx=None, tt=None):
        img, _ = O.render(cs, x if xx is None else xx, tex=tt)
        return float((img * dimg).sum())

    eps = 1e-6
    for k in range(12):
        xp, xm = x.copy(), x.copy()
        xp[0, k] += eps
        xm[0, k] -= eps
        fd = (fval(xp) - fval(xm)) / (2 * eps)
        assert abs(ds[0, k] - fd) <= 1e-5 * max(1.0, abs(fd)), (k, ds[0, k], fd)
    t0 = np.asarray(cs.textures, np.float64)
    for idx in [(0, 2, 3, 0), (0, 4, 1, 2), (0, 0, 0, 1)]:
        tp, tm = t0.copy(), t0.copy()
        tp[idx] += eps
        tm[idx] -= eps
        fd = (fval(tt=tp) - fval(tt=tm)) / (2 * eps)
        assert abs(dt[idx] - fd) <= 1e-5 * max(1.0, abs(fd)), (idx, dt[idx], fd)
