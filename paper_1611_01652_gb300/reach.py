"""Training a controller through the differentiable engine: the 4-degree-of-freedom arm reaching
for targets (section 3.2). One iteration is a batched rollout of the arm on every task of the
batch, the reverse pass for the controller gradient (the library's kernels), and an Adam step on
the controller weights, with the paper's training tricks: the objective is the distance to the
target averaged over the steps, the gradient decays by alpha per step (set on the model), the
controller starts from the zero policy, and the gradient's L2 norm is limited to 1.

The physics, its reverse mode and the Adam step run in the library's kernels; this module orders
the calls, scales the gradient to its norm limit, and reads the tips' final positions."""
from __future__ import annotations

import numpy as np

from .binding import World, ws_adam


class ReachTrainer:
    def __init__(self, model, lr=1e-3, clip=1.0):
        import torch

        self.model, self.lr, self.clip = model, float(lr), float(clip)
        self.world = World(model)
        self.W = torch.tensor(np.asarray(model.W, np.float32), device="cuda")
        self.dW = torch.zeros_like(self.W)
        self.m = torch.zeros_like(self.W)
        self.v = torch.zeros_like(self.W)
        self.loss = torch.zeros(model.B, device="cuda")
        self.dloss = torch.full((model.B,), 1.0 / model.B, device="cuda")  # gradient of the batch mean
        self.state = torch.zeros(model.B, model.nb, 18, device="cuda")
        self.t = 0

    def step(self):
        """One iteration; returns the batch-mean objective of the weights it started from (a
        device scalar)."""
        self.world.rollout(self.W, self.loss)
        self.world.backward(self.dloss, self.dW)
        norm = self.dW.norm()
        self.dW.mul_(self.clip / norm.clamp(min=self.clip))  # L2 norm at most `clip`
        self.t += 1
        ws_adam(self.W, self.dW, self.m, self.v, self.t, self.lr)
        return self.loss.mean()

    def final_distance(self):
        """Distance of every tip to its target at the end of a rollout with the current weights."""
        self.world.rollout(self.W, self.loss)
        self.world.get_state(self.state)
        self.world.sync()
        m = self.model
        x = self.state[:, m.loss_body].double().cpu().numpy()
        R = x[:, 3:12].reshape(-1, 3, 3)
        tip = x[:, 0:3] + np.einsum("bij,bj->bi", R, np.asarray(m.loss_point, np.float64))
        return np.linalg.norm(tip - np.asarray(m.loss_target, np.float64), axis=1)


def train(model, iters, lr0=3e-3, lr1=3e-4, clip=1.0, log_every=100):
    """Trains the model's controller for ``iters`` iterations of ReachTrainer, the learning rate
    decaying from ``lr0`` to ``lr1`` along a half cosine. Returns the logged (iteration, batch-mean
    objective) pairs and the tips' final distances to their targets before and after training."""
    import math

    tr = ReachTrainer(model, lr=lr0, clip=clip)
    before = tr.final_distance()
    hist = []
    for k in range(iters):
        tr.lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * k / iters))
        loss = tr.step()
        if k % log_every == 0 or k == iters - 1:
            hist.append((k, float(loss)))
    return hist, before, tr.final_distance()
