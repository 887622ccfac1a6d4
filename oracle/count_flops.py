"""Algorithmic FP32 work per simulated step of each workload, tallied by the
oracle's counting real type over rollouts drawn from the initial CE
distribution (mean = mid-bounds, cov = diag((range/4)^2)).  Writes
workload/flops_per_step.json, which the benchmark reads for its roofline.
Run: python oracle/count_flops.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workload  # noqa: E402


def tally(scene, skel, n=128, seed=1):
    lo, hi = np.array(skel["lo"]), np.array(skel["hi"])
    th = oracle.sample(seed, 0, 0, n, (lo + hi) / 2, np.diag((hi - lo) / 4))
    ops = oracle.count_ops(scene, skel, th)
    steps = ops.pop("steps")
    per = {k: v / steps for k, v in ops.items()}
    per["flops"] = per["add"] + per["mul"]
    return per


def main():
    out = {}
    for cfg in (0, 1, 2):
        sc, sk, cm = workload.config(cfg, seed=0)
        out[cm["name"]] = dict(tally(sc, sk), N=cm["N"], T=sc["T"], D=len(sk["lo"]),
                               samples=128, distribution="initial")
    path = os.path.join(ROOT, "workload", "flops_per_step.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
