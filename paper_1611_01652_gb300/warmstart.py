"""Learned warm start of the solver: harvest of training rows from rollouts and training of the
16-64-64-3 network, every step on the GPU through the library's C ABI (dp_harvest,
dp_ws_loss_grad, dp_ws_adam). This module only orders the calls.

A harvested row holds the 16 features of an active row group before the solve and the network's
ideal output: the impulses the solve reached minus alpha times the previous step's. Harvesting
worlds solve with many sweeps so that these impulses are close to converged. Gait perturbations
are seeded Gaussian noise added to the controller output at every step.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as _b

WS_IN, WS_H, WS_OUT = 16, 64, 3
WS_PARAMS = WS_IN * WS_H + WS_H + WS_H * WS_H + WS_H + WS_H * WS_OUT + WS_OUT


def init_params(seed=0, out_scale=1.0):
    """Xavier-uniform weights, zero biases, flat layout W1, b1, W2, b2, W3, b3 (numpy float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ni, no) in enumerate(((WS_IN, WS_H), (WS_H, WS_H), (WS_H, WS_OUT))):
        a = math.sqrt(6.0 / (ni + no)) * (out_scale if i == 2 else 1.0)
        parts.append(rng.uniform(-a, a, size=(no, ni)).reshape(-1))
        parts.append(np.zeros(no))
    W = np.concatenate(parts).astype(np.float32)
    assert W.size == WS_PARAMS
    return W


def harvest(world, W, max_rows, noise_sigma=0.1, seed=0):
    """Rows [n, 19] (device tensor) from one rollout of ``world`` (with its current solver) with
    controller weights W and N(0, noise_sigma) perturbations of every controller output."""
    import torch

    dev = torch.device("cuda")
    rows = torch.empty(int(max_rows), _b.WS_ROW, device=dev, dtype=torch.float32)
    noise = None
    if noise_sigma > 0 and world.n_motors > 0:
        g = torch.Generator(device=dev)
        g.manual_seed(int(seed))
        noise = torch.randn(world.horizon, world.B, world.n_motors, device=dev, generator=g) * float(noise_sigma)
    n = world.harvest(W, rows, noise)
    return rows[:n]


def feature_scaling(rows):
    """Per-feature mean and spread of harvested rows (device [n, 19]); the spread is floored so
    that nearly constant features are not blown up."""
    import torch

    x = rows[:, :WS_IN].double()
    mu = x.mean(0)
    sd = torch.maximum(x.std(0), 0.1 * mu.abs() + 1e-2)
    return mu.float(), sd.float()


def fold_scaling(W, mu, sd):
    """Parameters of the network on raw features from those of the network on standardised
    features (x - mu) / sd: W1' = W1 / sd, b1' = b1 - W1' mu."""
    W = W.clone()
    W1 = W[:WS_IN * WS_H].view(WS_H, WS_IN)
    b1 = W[WS_IN * WS_H:WS_IN * WS_H + WS_H]
    W1s = W1 / sd[None, :]
    b1 -= (W1s * mu[None, :]).sum(1)
    W1.copy_(W1s)
    return W


def train(rows, steps=2000, batch=65536, lr=2e-3, seed=0, W0=None, val_rows=None, log_every=0, standardise=True,
          finetune=200):
    """Adam on the mean squared error over minibatches of ``rows`` (device [n, 19]). With
    ``standardise`` the network first learns on standardised features, its first layer is then
    folded back to raw features and ``finetune`` steps adapt it to the bfloat16 rounding of the
    raw inputs. Returns the trained parameters on raw features (device float32 [WS_PARAMS]) and the
    loss history [(step, train, val)] (val on raw features)."""
    import torch

    dev = rows.device
    n = rows.shape[0]
    batch = int(min(batch, n))
    W = torch.tensor(init_params(seed) if W0 is None else W0, device=dev, dtype=torch.float32)
    work = _b.ws_workspace(max(batch, val_rows.shape[0] if val_rows is not None else 0), device=dev)
    mu = sd = None
    src = rows
    if standardise:
        mu, sd = feature_scaling(rows)
        src = rows.clone()
        src[:, :WS_IN] = (src[:, :WS_IN] - mu) / sd
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) + 1)
    hist = []

    def run(data, W, nsteps, lr0, step0):
        m = torch.zeros_like(W)
        v = torch.zeros_like(W)
        dW = torch.zeros_like(W)
        loss = torch.zeros(1, device=dev)
        perm = torch.randperm(n, device=dev, generator=g)
        pos = 0
        for it in range(1, nsteps + 1):
            if pos + batch > n:
                perm = torch.randperm(n, device=dev, generator=g)
                pos = 0
            mb = data.index_select(0, perm[pos:pos + batch]).contiguous()
            pos += batch
            _b.ws_loss_grad(W, mb, loss, dW, work)
            lr_t = lr0 * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / nsteps))  # cosine decay
            _b.ws_adam(W, dW, m, v, it, lr_t)
            if log_every and (it % log_every == 0 or it == nsteps):
                Wr = fold_scaling(W, mu, sd) if (standardise and data is src and src is not rows) else W
                vl = evaluate(Wr, val_rows, work) if val_rows is not None else None
                hist.append((step0 + it, float(loss.item()), vl))
        return W

    W = run(src, W, steps, lr, 0)
    if standardise:
        W = fold_scaling(W, mu, sd)
        if finetune:
            W = run(rows, W, finetune, lr * 0.1, steps)
    return W, hist


def shrink(W, kappa):
    """The network with its output scaled by kappa (the linear output layer W3, b3 times kappa):
    its correction to the damped start is kappa times the original's."""
    W = W.clone()
    n3 = WS_H * WS_OUT + WS_OUT
    W[-n3:] *= float(kappa)
    return W


def evaluate(W, rows, work=None):
    """Mean squared error of the network W over rows (device [n, 19])."""
    import torch

    work = work if work is not None else _b.ws_workspace(rows.shape[0], device=rows.device)
    loss = torch.zeros(1, device=rows.device)
    dW = torch.zeros(WS_PARAMS, device=rows.device)
    _b.ws_loss_grad(W, rows.contiguous(), loss, dW, work)
    return float(loss.item())


def _rollout_residual(model, iters, net, alpha, W, horizon):
    """Mean per-step solve residual of one rollout (None if it produced a non-finite value)."""
    import torch

    from .binding import DPError, World

    w = World(model, horizon=horizon, iters=iters, warmstart=True)
    if net is not None:
        w.set_warmstart(net, alpha)
    w.set_residual(True)
    loss = torch.zeros(model.B, device="cuda")
    w.rollout(W, loss)
    r = torch.zeros(model.B, device="cuda")
    w.get_residual(r)
    try:
        w.sync()
    except DPError:
        return None
    v = float(r.mean().item())
    return v if math.isfinite(v) else None


def _one_step_states(model, iters, net, alpha, W, x, lam_prev, t):
    """One step from states x [B, nb, 18] and previous impulses: next states [B, nb, 18]."""
    import torch

    from .binding import World

    w = World(model, horizon=1, iters=iters, warmstart=True)
    if net is not None:
        w.set_warmstart(net, alpha)
    w.set_state(x, t)
    w.set_impulses(lam_prev)
    w.step(1, W)
    out = torch.zeros_like(x)
    w.get_state(out)
    w.sync()
    return out


def _controller_gradient(model, iters, net, alpha, W, horizon):
    import torch

    from .binding import World

    w = World(model, horizon=horizon, iters=iters, warmstart=True)
    if net is not None:
        w.set_warmstart(net, alpha)
    loss = torch.zeros(model.B, device="cuda")
    w.rollout(W, loss)
    dW = torch.zeros(w.n_params, device="cuda")
    w.backward(torch.ones(model.B, device="cuda"), dW)
    w.sync()
    return dW


def accept(model, candidates, plain_iters=20, sweep_grid=(5, 7, 10, 14), horizon=200, ref_iters=80, state_tol=1e-3,
           grad_tol=2e-2):
    """Acceptance gate of warm starts against the plain cold-start solver at ``plain_iters``
    sweeps on held-out robots (``model``; its controller weights drive them). State and gradient
    errors are measured against the plain solver at ``ref_iters`` sweeps.

    For each candidate (name, network parameters, alpha), at the smallest sweep count N of the
    grid where it gets there, the warm-started solver must (1) stay finite over a
    ``horizon``-step rollout with a mean solve residual no larger than the plain solver's,
    (2) make one-step state errors (from the reference rollout's states and impulses at a few
    times; relative, scale floor 1) at most ``state_tol`` above the plain solver's, and (3) make
    a 10-step controller-gradient error (relative norm) at most ``grad_tol`` above the plain
    solver's. Returns a report dict; ``report["accepted"]`` is the accepted (name, N, alpha) with
    the fewest sweeps (ties: the lower residual), or None (the plain solver is then used);
    ``report["accepted_all"]`` lists every accepted (name, N, alpha) in that order."""
    import torch

    from .binding import World

    W = torch.tensor(model.W, device="cuda")
    rep = {"plain_iters": plain_iters, "ref_iters": ref_iters,
           "plain_resid": _rollout_residual(model, plain_iters, None, 0.0, W, horizon), "candidates": []}
    wp = World(model, horizon=horizon, iters=ref_iters, warmstart=True)
    traj = torch.zeros(horizon + 1, model.B, model.nb, 18, device="cuda")
    wp.rollout(W, torch.zeros(model.B, device="cuda"), traj)
    wp.sync()
    times = [horizon // 4, horizon // 2, horizon - 1]
    lams = {}
    for t in times:
        wt = World(model, horizon=t, iters=ref_iters, warmstart=True)
        wt.rollout(W, torch.zeros(model.B, device="cuda"))
        lam = torch.zeros(model.B, wt.n_slots, device="cuda")
        wt.get_impulses(lam)
        wt.sync()
        lams[t] = lam

    def state_err(iters, net, alpha):
        e = 0.0
        for t in times:
            x = traj[t].contiguous()
            ref = _one_step_states(model, ref_iters, None, 0.0, W, x, lams[t], t)
            xn = _one_step_states(model, iters, net, alpha, W, x, lams[t], t)
            e = max(e, float(((xn - ref).abs() / ref.abs().clamp_min(1.0)).max().item()))
        return e

    g_ref = _controller_gradient(model, ref_iters, None, 0.0, W, 10)

    def grad_err(iters, net, alpha):
        g = _controller_gradient(model, iters, net, alpha, W, 10)
        return float(((g - g_ref).norm() / g_ref.norm().clamp_min(1e-30)).item())

    rep["plain_state_err"] = state_err(plain_iters, None, 0.0)
    rep["plain_grad_err"] = grad_err(plain_iters, None, 0.0)
    for name, net, alpha in candidates:
        for N in sorted(sweep_grid):
            if N >= plain_iters:
                break
            r = _rollout_residual(model, N, net, alpha, W, horizon)
            entry = {"name": name, "alpha": alpha, "iters": N, "resid": r}
            if r is None or rep["plain_resid"] is None or r > rep["plain_resid"]:
                entry["accepted"] = False
                rep["candidates"].append(entry)
                continue
            entry["state_err"] = state_err(N, net, alpha)
            entry["grad_err"] = grad_err(N, net, alpha)
            entry["accepted"] = bool(entry["state_err"] <= rep["plain_state_err"] + state_tol and
                                     entry["grad_err"] <= rep["plain_grad_err"] + grad_tol)
            rep["candidates"].append(entry)
            break  # the smallest sweep count at which this candidate reaches the plain residual
    ok = sorted((c for c in rep["candidates"] if c["accepted"]), key=lambda c: (c["iters"], c["resid"]))
    rep["accepted_all"] = [(c["name"], c["iters"], c["alpha"]) for c in ok]
    rep["accepted"] = rep["accepted_all"][0] if ok else None
    return rep
