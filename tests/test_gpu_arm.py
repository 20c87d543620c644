"""The 4-degree-of-freedom arm of section 3.2 through the C ABI against the FP64 oracle: two
universal joints composed of hinge pairs with a cross body, four servos driven by the
11-64-64-4 controller with a non-zero output layer (so that every joint moves), no gravity, the
per-step averaged tip distance and the gradient decay of 0.5 (section 3.2). Free-running
rollouts within 1e-4 over the first 80 steps and 1e-3 over 100 (the 2 kg cross bodies between
14 kg links, driven by 30 1/s servos, amplify the fp32 rounding in the last steps, as the long
pendulum rollout does), and the gradients with respect to the initial state, the
masses, the servo parameters and every controller weight over 60 steps, element by element
within 1e-3 (fp32 controller, so that no bfloat16 rounding decision differs)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1611_01652_gb300 import workloads as WL  # noqa: E402

from test_gpu_parity import GRAD_RTOL, check_grads, compare_rollout, elem_err  # noqa: E402

pytestmark = pytest.mark.gpu


def moving_arm(B, horizon):
    m = WL.arm4dof(B=B, horizon=horizon)
    m.ctrl_fp32 = 1
    rng = np.random.default_rng(5)
    W = np.asarray(m.W, np.float32).copy()
    n3 = m.widths[2] * m.widths[3] + m.widths[3]
    W[-n3:] = rng.uniform(-0.5, 0.5, size=n3).astype(np.float32)  # the servos move
    m.W = W
    return m


def test_arm_rollout_matches_oracle():
    m = moving_arm(8, 100)
    compare_rollout(m, 100, range(8), min_clean=1.0, rtol=1e-3, rtol_window=(80, 1e-4))


def test_arm_gradients_match_oracle():
    m = moving_arm(4, 60)
    assert m.grad_decay == 0.5
    g, Wsum = check_grads(m, 60, ("state0", "mass", "motor", "anchor"), range(4), with_W=True)
    assert elem_err(g["W"], Wsum) <= GRAD_RTOL
    assert np.abs(g["W"]).max() > 0
