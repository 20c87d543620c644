"""Writes tests/golden/flops_per_instance_step.json: the algorithmic operation count of one
instance-step of each workload, from the oracle's instrumented counter (forward: every
arithmetic operation and elementary function; reverse: one multiply and one add per partial
derivative recorded on the reverse-mode tape). Averaged over seeded instances and steps.

Calls only the oracle and the seeded workload generators. Run: python -m oracle.flop_counts
"""
import json
import os

import numpy as np

import oracle as O
from paper_1611_01652_gb300 import workloads as WL

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "flops_per_instance_step.json")


def average(m, instances, horizon):
    acc = np.zeros(3)
    for i in instances:
        acc += np.array(O.flops(m, i, horizon))
    return acc / len(instances)


def main():
    res = {"_about": "Algorithmic operations per instance-step from the FP64 oracle's instrumented counter "
                     "(oracle/flop_counts.py); forward = counted arithmetic, reverse = 2 per recorded partial."}
    cases = {
        "quadruped_b4096_t1000": (WL.quadruped(B=8, horizon=200), range(8), 200),
        "pendulum3_b1024_t1000": (WL.pendulum3(B=8, horizon=200), range(8), 200),
        "ball_b1_t300": (WL.ball(B=8, horizon=300), range(8), 300),
    }
    for n in (5, 7, 10, 14):  # the solve at fewer sweeps (a warm-started solver's counts)
        cases["quadruped_b4096_t1000_iters%d" % n] = (WL.quadruped(B=8, horizon=200, iters=n), range(8), 200)
    for name, (m, inst, T) in cases.items():
        f, r, n = average(m, inst, T)
        res[name] = {"forward": round(float(f), 1), "reverse": round(float(r), 1), "tape_nodes": round(float(n), 1),
                     "instances": len(inst), "steps": T}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=2)
    print(json.dumps(res, indent=2))


if __name__ == "__main__":
    main()
