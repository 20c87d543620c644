"""System identification through the differentiable engine: per-instance model parameters fitted
by gradient descent so that the simulated motion reproduces observations (the paper's outlook:
optimise model parameters with gradient descent through physics until the model mimics the
measurements). Every system of a batch (one instance, or K instances that are K experiments on
one system) is its own identification problem; one iteration is a batched rollout, the reverse
pass for the parameter gradients, and one Adam step.

The physics, its reverse mode and the Adam steps run in the library's kernels; this module orders
the calls, sums the gradients of experiments that share a system, and keeps the iterates inside
the parameters' physical ranges.
"""
from __future__ import annotations

import numpy as np

from .binding import World, ws_adam

# physical range of each fitted group (clamped after every step)
RANGES = {"sph_e": (0.0, 1.0), "sph_mu": (0.0, 2.0), "mass": (1e-3, None), "inertia": (1e-6, None),
          "sph_rad": (1e-3, None)}


def observe(model, truth):
    """World position [B, 3] of the model's loss point (a point fixed on its loss body) at the
    final step of a rollout with the parameter groups ``truth`` (dict of arrays) in place of the
    model's own: the observations of a fit."""
    import torch

    w = World(model)
    w.set_params(**truth)
    traj = torch.zeros(w.horizon + 1, model.B, model.nb, 18, device="cuda")
    w.rollout(None, torch.zeros(model.B, device="cuda"), traj)
    w.sync()
    x = traj[-1, :, model.loss_body].double().cpu().numpy()
    R = x[:, 3:12].reshape(-1, 3, 3)
    c = np.asarray(model.loss_point, np.float64)
    return torch.tensor(x[:, 0:3] + np.einsum("bij,bj->bi", R, c), dtype=torch.float32, device="cuda")


class Fit:
    """Adam on the parameter groups ``names``, the loss being the model's own squared distance of
    its loss point at the final step to ``observed`` [B, 3] (its loss target). With ``shared`` = K,
    consecutive runs of K instances are K experiments on one system: they share one value of each
    parameter, whose gradient is the sum of theirs."""

    def __init__(self, model, observed, names=("mass",), lr=0.01, shared=1):
        import torch

        assert model.B % shared == 0
        self.model, self.names, self.lr, self.K = model, tuple(names), float(lr), int(shared)
        self.world = World(model)
        self.world.set_params(loss_target=observed.contiguous())
        per = {k: torch.tensor(np.asarray(getattr(model, k), np.float32), device="cuda") for k in self.names}
        # one value per system (the first experiment's), expanded to its K instances when set
        self.p = {k: v[::self.K].contiguous() for k, v in per.items()}
        self.inst = {k: v.clone() for k, v in per.items()}
        self.g = {k: torch.zeros_like(v) for k, v in per.items()}
        self.gs = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.loss = torch.zeros(model.B, device="cuda")
        self.dloss = torch.ones(model.B, device="cuda")
        self.t = 0

    def _expand(self):
        for k in self.names:
            self.inst[k].view(-1, self.K, *self.p[k].shape[1:]).copy_(self.p[k].unsqueeze(1))
        self.world.set_params(**self.inst)

    def step(self):
        """One iteration: set the parameters, roll out, reverse pass, Adam; returns the per-instance
        loss of the parameters the iteration started from (a device tensor)."""
        import torch

        self._expand()
        self.world.rollout(None, self.loss)
        for g in self.g.values():
            g.zero_()
        self.world.backward(self.dloss, None, None, self.g)
        self.t += 1
        for k in self.names:
            torch.sum(self.g[k].view(-1, self.K, *self.p[k].shape[1:]), 1, out=self.gs[k])
            ws_adam(self.p[k], self.gs[k], self.m[k], self.v[k], self.t, self.lr)
            lo, hi = RANGES.get(k, (None, None))
            self.p[k].clamp_(min=lo, max=hi)
        return self.loss

    def run(self, iters):
        for _ in range(iters):
            self.step()
        self._expand()
        self.world.rollout(None, self.loss)
        self.world.sync()
        return self.loss
