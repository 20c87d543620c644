#!/usr/bin/env python3
"""Throughput of batched differentiable rigid-body rollouts (arXiv 1611.01652) on GB300.

One step = one forward rollout plus its full reverse-mode gradient (dp_rollout + dp_backward)
of the quadruped batch: B = 4096 instances, T = 1000 steps of 10 ms, 20 solver sweeps, dense
controller 24->128->128->8 (bfloat16 weights, fp32 accumulation), loss = negative forward
displacement, gradient w.r.t. every controller weight. Metric: instance-steps/s (B*T per step).

Prints one JSON line. `--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inst-steps/s fwd+adjoint, quadruped B=4096; warm-start vs plain @equal resid"
FLOPS = os.path.join(ROOT, "tests", "golden", "flops_per_instance_step.json")
SM_COUNT, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=4096)
    p.add_argument("--horizon", type=int, default=1000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------------------ CPU oracle legs
def _oracle_worker(args):
    n_inst, horizon, seed = args
    import oracle as O
    from paper_1611_01652_gb300 import workloads as WL

    m = WL.quadruped(B=n_inst, horizon=horizon, seed=seed)
    t0 = time.perf_counter()
    for i in range(n_inst):
        O.rollout_grad(m, i, horizon=horizon)
    return time.perf_counter() - t0


def oracle_sample(workers, n_inst, horizon):
    """Forward+adjoint of the quadruped on the FP64 oracle, `workers` processes (spawned) each
    doing `n_inst` instances x `horizon` steps. Returns (inst-steps/s, seconds, inst-steps)."""
    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_worker, [(1, 2, 5000 + k) for k in range(workers)])  # warm the processes
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [(n_inst, horizon, 6000 + k) for k in range(workers)])
        dt = time.perf_counter() - t0
    units = workers * n_inst * horizon
    return units / dt, dt, units


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank):
    if rank != 0:
        return
    cores = min(host_cores(), 16)
    vals = []
    for k in range(args.warmup + args.steps):
        v, dt, units = oracle_sample(cores, 1, 60)
        if k >= args.warmup:
            vals.append((v, dt, units))
    value = statistics.median(v for v, _, _ in vals)
    ms = statistics.median(dt for _, dt, _ in vals) * 1e3
    sample = "per step: %d processes x 1 instance x 60 steps of the quadruped forward+adjoint (FP64 oracle)" % cores
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "inst-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "quadruped B=4096 T=1000 iters=20, MLP 24-128-128-8, fwd+adjoint (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "inst-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "inst-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch

    from paper_1611_01652_gb300 import workloads as WL
    from paper_1611_01652_gb300.binding import World

    torch.cuda.set_device(local_rank)
    dist = None
    if world_size > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    B, T = args.batch, args.horizon
    m = WL.quadruped(B=B, horizon=T, seed=1002 + 17 * rank)
    stream = torch.cuda.current_stream()
    world = World(m, stream=stream)
    W = torch.tensor(m.W, device="cuda")
    loss = torch.empty(B, device="cuda")
    dloss = torch.ones(B, device="cuda")
    dW = torch.empty(world.n_params, device="cuda")

    def step():
        world.rollout(W, loss)
        world.backward(dloss, dW)

    for _ in range(args.warmup):
        step()
    world.sync()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        world.rollout(W, loss)
        ev[k][1].record(stream)
        world.backward(dloss, dW)
        ev[k][2].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    world.sync()
    total_ms = t0.elapsed_time(t1)
    fwd_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    bwd_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    if dist:
        tt = torch.tensor([total_ms, fwd_ms, bwd_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms, fwd_ms, bwd_ms = tt.tolist()
    ms_per_step = total_ms / args.steps
    value = B * T * world_size / (ms_per_step / 1e3)

    # end to end through the C ABI with host buffers (pinned): W and dloss in, loss and dW out
    e2e = None
    if not args.no_e2e:
        Wh = torch.tensor(m.W).pin_memory()
        dlh = torch.ones(B).pin_memory()
        lh = torch.empty(B).pin_memory()
        dWh = torch.empty(world.n_params).pin_memory()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            world.rollout(Wh, lh)
            world.backward(dlh, dWh)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / args.steps
        if dist:
            tt = torch.tensor([ems], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ems = tt.item()
        e2e = {"value": B * T * world_size / (ems / 1e3), "unit": "inst-steps/s",
               "h2d_bytes_per_step": 4 * (world.n_params + B), "d2h_bytes_per_step": 4 * (B + world.n_params)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fl = json.load(open(FLOPS))["quadruped_b4096_t1000"]
    peak = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12  # TFLOP/s, FP32 FMA at max SM clock
    achieved = fl["reverse"] * B * T / (bwd_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_backward", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "basis": "reverse-mode algorithmic FP ops per instance-step (oracle counter) x B x T / dp_backward time; "
                         "peak = 152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived; no measured FP32 peak)",
                "step_frac": (fl["forward"] + fl["reverse"]) * B * T / (ms_per_step / 1e3) / 1e12 / peak}
    cpu = None
    if not args.no_cpu_baseline and world_size == 1:
        cores = min(host_cores(), 16)
        v, dt, units = oracle_sample(cores, 2, 100)
        cpu = {"value": v, "unit": "inst-steps/s", "cores": cores, "kind": "oracle",
               "sample": "%d spawned processes x 2 quadruped instances x 100 steps, forward+adjoint, FP64 oracle "
                         "(%.1f s wall)" % (cores, dt)}
    n_dense = len(m.widths) - 1 + (1 if m.skip else 0)
    launches_per_step = 2 + 2 + 4 * n_dense  # prep+forward; pad+backward; per dense layer: gemm, sum, rowsum, sum
    out = {
        "metric": METRIC, "value": value, "unit": "inst-steps/s", "n_gpus": world_size, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "quadruped B=%d T=%d iters=20, MLP 24-128-128-8 (bf16 weights, fp32 acc), "
                               "forward+adjoint, gradient w.r.t. all controller weights" % (B, T),
                   "batch": B, "horizon": T, "iters": m.iters, "ckpt_every": world.ckpt_every,
                   "l2": "working set (checkpoints + controller activations) >> 129 MB L2; no flush needed"},
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": ck,
        "gpu_launches": launches_per_step * args.steps, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
        "loss_mean": float(loss.mean().item()), "finite": bool(torch.isfinite(dW).all().item()),
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
