"""Pin of the 4-degree-of-freedom arm's universal joints (two hinges with perpendicular axes
meeting in one point, a cross body between them) on the oracle: while a random controller
drives all four servos, every relative rotation stays a rotation about its hinge axis alone and
the tip sits where the closed-form forward kinematics of the four joint angles puts it, both up
to the drift the soft constraints allow (5e-3; no GPU)."""
import numpy as np

import oracle as O
from paper_1611_01652_gb300 import workloads as WL


def rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def ry(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rx(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def test_composed_universal_joints_follow_forward_kinematics():
    m = WL.arm4dof(B=4, horizon=300)
    rng = np.random.default_rng(5)
    W = np.asarray(m.W, np.float64).copy()
    n3 = m.widths[2] * m.widths[3] + m.widths[3]
    W[-n3:] = rng.uniform(-0.5, 0.5, size=n3)  # a non-zero output layer: the servos move
    moved = 0.0
    for i in range(4):
        st = O.rollout(m, i, W=W)[0]
        for t in range(0, 301, 30):
            R = [st[t, b, 3:12].reshape(3, 3) for b in range(4)]
            th0 = np.arctan2(R[0][1, 0], R[0][0, 0])
            assert np.abs(R[0] - rz(th0)).max() <= 5e-3, (i, t)
            rel = [R[0].T @ R[1], R[1].T @ R[2], R[2].T @ R[3]]
            th1 = np.arctan2(rel[0][0, 2], rel[0][0, 0])
            th2 = np.arctan2(rel[1][0, 2], rel[1][0, 0])
            th3 = np.arctan2(rel[2][2, 1], rel[2][1, 1])
            assert np.abs(rel[0] - ry(th1)).max() <= 5e-3, (i, t)
            assert np.abs(rel[1] - ry(th2)).max() <= 5e-3, (i, t)
            assert np.abs(rel[2] - rx(th3)).max() <= 5e-3, (i, t)
            tip_fk = rz(th0) @ ry(th1) @ (np.array([0.0, 0.0, 0.5]) + ry(th2) @ rx(th3) @ np.array([0.0, 0.0, 0.5]))
            tip = st[t, 3, 0:3] + R[3] @ np.array([0.0, 0.0, 0.25])
            assert np.abs(tip - tip_fk).max() <= 5e-3, (i, t, tip, tip_fk)
            moved = max(moved, abs(th0), abs(th1), abs(th2), abs(th3))
    assert moved > 0.2


def test_reach_gradient_matches_central_differences():
    """The reaching objective (distance to the target averaged over the steps) of the arm under a
    non-zero controller: its reverse-mode gradient w.r.t. controller weights equals central
    differences of the oracle's forward pass (no decay, controller unrounded; outputs small
    enough that no servo reaches its rate limit, a kink of the objective)."""
    from test_oracle_pins import _same_activity

    m = WL.arm4dof(B=2, horizon=40, grad_decay=1.0)
    m.exact_mlp = 1
    rng = np.random.default_rng(8)
    W = np.asarray(m.W, np.float64).copy()
    n3 = m.widths[2] * m.widths[3] + m.widths[3]
    W[-n3:] = rng.uniform(-0.02, 0.02, size=n3)
    L, g = O.rollout_grad(m, 0, W=W)
    n1 = m.widths[0] * m.widths[1]
    checked = 0
    for k in [3, 40, n1 - 5, n1 + 64 + 100, len(W) - n3 + 5, len(W) - 3, len(W) - 1]:
        eps = 1e-6
        Wp, Wm = W.copy(), W.copy()
        Wp[k] += eps
        Wm[k] -= eps
        if not _same_activity(m, 0, m.horizon, None, None, Wp, Wm):
            continue
        fd = (O.rollout(m, 0, W=Wp)[1] - O.rollout(m, 0, W=Wm)[1]) / (2 * eps)
        assert abs(fd - g["W"][k]) <= 1e-4 * (abs(fd) + 1e-4), (k, fd, g["W"][k])
        checked += 1
    assert checked >= 5
