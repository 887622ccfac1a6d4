"""Algorithmic FP32 work per simulated step of each workload, tallied by the
oracle's counting real type over rollouts drawn from the initial CE
distribution (mean = mid-bounds, cov = diag((range/4)^2)); for the
64-problem batch, per problem.  Writes
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


def batch_tally(seed=0, n=64):
    """Per problem of the 64-problem batch (workload.batch_problems(seed)):
    flops per step over n samples of its initial distribution, plus the
    mean per skeleton length weighted by each problem's N x T."""
    per, by_len = [], {}
    for p in workload.batch_problems(seed):
        t = tally(p["scene"], p["skel"], n=n)
        per.append(dict(L=p["L"], N=p["N"], T=p["scene"]["T"], D=len(p["skel"]["lo"]), flops=t["flops"],
                        div=t["div"], sqrt=t["sqrt"], transc=t["transc"]))
        w = p["N"] * p["scene"]["T"]
        acc = by_len.setdefault(str(p["L"]), [0.0, 0.0])
        acc[0] += w * t["flops"]
        acc[1] += w
    return dict(seed=seed, samples_per_problem=n, distribution="initial", problems=per,
                flops_by_length={L: v[0] / v[1] for L, v in sorted(by_len.items())})


def main():
    out = {}
    for cfg in (0, 1, 2):
        sc, sk, cm = workload.config(cfg, seed=0)
        out[cm["name"]] = dict(tally(sc, sk), N=cm["N"], T=sc["T"], D=len(sk["lo"]),
                               samples=128, distribution="initial")
    out["batch-64"] = batch_tally()
    path = os.path.join(ROOT, "workload", "flops_per_step.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
