"""Uneven batches: robots of several topologies and horizons in one forward + adjoint pass.

Instances are binned by topology (one World per bin, since a world's kernels are specialised
to one topology); inside a bin they are ordered by horizon, longest first, so that the 32
instances of a warp have similar horizons and each warp steps only to its own longest one. Each
bin gets the launch configuration an autotuner picked by timing short rollouts: the mapping of
a group of 32 instances (four warps, with the compiled topology's kernels, or one warp),
constraint rows on chip or in global memory, whole solver tape or checkpoint segments, split
count of the controller-gradient reduction. All bins run concurrently, each on its own stream, and the
whole pass (every bin's rollout and reverse pass, and the sum of the controller gradients) can
be captured once as a CUDA graph and replayed as a single launch.

All arithmetic runs in the library's kernels; this module only orders calls.
"""
from __future__ import annotations

import itertools

import numpy as np

from .binding import World


def _order_by_horizon(m):
    """The bin's instances sorted by horizon (longest first); returns the reordered model and
    the permutation."""
    perm = np.argsort(-np.asarray(m.horizons), kind="stable")
    return m.subset(perm), perm


# one warp per group of 32 instances with every row/tape/split choice; four warps per group (the
# compiled topologies' kernels, which keep the rows on chip and the whole tape) with each split
CANDIDATES = ([dict(rows_global=rg, ckpt_every=ck, dw_splits=sp, one_warp=True)
               for rg, ck, sp in itertools.product((False, True), (0, 16), (64, 256))] +
              [dict(rows_global=False, ckpt_every=0, dw_splits=sp, one_warp=False) for sp in (64, 256)])


def autotune(m, W, horizon=64, reps=2, candidates=None, stream=None):
    """Times a short rollout + reverse pass of bin ``m`` (its first ``horizon`` steps) for each
    launch configuration and returns (best configuration, [(configuration, ms)])."""
    import torch

    res = []
    short = m.subset(np.arange(m.B))
    short.horizons = np.minimum(np.asarray(m.horizons), horizon).astype(np.int32)
    s = stream or torch.cuda.current_stream()
    for cfg in candidates or CANDIDATES:
        w = World(short, stream=stream, horizon=horizon, ckpt_every=cfg["ckpt_every"], rows_global=cfg["rows_global"],
                  dw_splits=cfg["dw_splits"], one_warp=cfg["one_warp"])
        loss = torch.zeros(short.B, device="cuda")
        dl = torch.ones(short.B, device="cuda")
        dW = torch.zeros(w.n_params, device="cuda")
        w.rollout(W, loss)
        w.backward(dl, dW)
        w.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            w.rollout(W, loss)
            w.backward(dl, dW)
        e1.record(s)
        w.sync()
        res.append((cfg, e0.elapsed_time(e1) / reps))
        del w
    best = min(res, key=lambda r: r[1])[0]
    return best, res


class UnevenBatch:
    """Forward + adjoint of an uneven batch given as {key: Model} bins (each with per-instance
    ``horizons``). ``tune`` picks each bin's launch configuration with ``autotune``."""

    def __init__(self, bins, W, tune=True, tune_horizon=64, iters=None):
        import torch

        self.W = W
        self.keys = sorted(bins)
        self.streams = {k: torch.cuda.Stream() for k in self.keys}
        self.models, self.perm, self.worlds, self.config, self.tuning = {}, {}, {}, {}, {}
        for k in self.keys:
            m, perm = _order_by_horizon(bins[k])
            if iters is not None:
                m.iters = iters
            self.models[k], self.perm[k] = m, perm
            if tune:
                best, res = autotune(m, W, horizon=tune_horizon, stream=self.streams[k])
                self.tuning[k] = res
            else:
                best = dict(rows_global=False, ckpt_every=0, dw_splits=0, one_warp=False)
            self.config[k] = best
            self.worlds[k] = World(m, stream=self.streams[k], ckpt_every=best["ckpt_every"],
                                   rows_global=best["rows_global"], dw_splits=best["dw_splits"],
                                   one_warp=best["one_warp"])
        n_params = self.worlds[self.keys[0]].n_params
        self.loss = {k: torch.zeros(self.models[k].B, device="cuda") for k in self.keys}
        self.dloss = {k: torch.ones(self.models[k].B, device="cuda") for k in self.keys}
        self.dW_bin = {k: torch.zeros(n_params, device="cuda") for k in self.keys}
        self.dW = torch.zeros(n_params, device="cuda")
        self.instance_steps = int(sum(int(np.sum(self.models[k].horizons)) for k in self.keys))
        self.graph = None

    def _issue(self):
        """Every bin's rollout and reverse pass on its own stream, joined on the current stream,
        then the sum of the bins' controller gradients."""
        import torch

        main = torch.cuda.current_stream()
        for k in self.keys:
            s = self.streams[k]
            s.wait_stream(main)
            with torch.cuda.stream(s):
                w = self.worlds[k]
                w.rollout(self.W, self.loss[k])
                w.backward(self.dloss[k], self.dW_bin[k])
        for k in self.keys:
            main.wait_stream(self.streams[k])
        torch.sum(torch.stack([self.dW_bin[k] for k in self.keys]), 0, out=self.dW)

    def run(self):
        """One forward + adjoint pass (eager, or the captured graph once captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._issue()
        return self.dW

    def capture(self):
        """Captures the whole pass as one CUDA graph (after one eager pass that warms it up)."""
        import torch

        self._issue()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._issue()
        torch.cuda.synchronize()
        self.graph = g

    def losses(self):
        """Per-instance losses in the bins' original instance order: {key: [B_k]}."""
        out = {}
        for k in self.keys:
            v = np.empty(self.models[k].B, np.float32)
            v[self.perm[k]] = self.loss[k].cpu().numpy()
            out[k] = v
        return out
