"""Benchmark of the CE plan-realization hot path on GB300.

One step = one cross-entropy iteration of Algorithm 1 for the 64-problem
batch (skeletons of 1..6 actions, N per problem log-uniform in [512, 8192],
T = 400 / 1000 / 3000, 4.5e8 simulated steps per iteration): the batched
Philox sampler -> ONE persistent rollout launch -> the segmented select +
refit, replayed from a CUDA graph, all on the device through the C ABI.
The timed steps are iterations 0..K-1 of one CE run from the initial
distributions.  Reported value: simulated steps per second (sum of N x T
over problems / time per iteration).  The single-problem move-and-push and
pick-place workloads are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs an independent replica (its own Philox
problem ids) on its own GPU: weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload  # noqa: E402

METRIC = "sim steps/sec (N×T) on 1 GB300 & FP32-peak fraction; CEM time-to-cost vs plain"
UNIT = "sim-steps/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SATURATED_N = 48 * 4096  # enough rollouts to give every SM scheduler several warps
CPU_FRACTION = 4  # the CPU legs roll out 1 / CPU_FRACTION of every problem's samples per iteration
REF_FRACTION = 8  # the reference arm: 1 / REF_FRACTION per step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rollout-only", choices=["reach", "push", "pickplace"], default=None,
                    help="time only the rollout kernel of one workload (profiling driver)")
    ap.add_argument("--n", type=int, default=0,
                    help="samples for --rollout-only (0 = the workload's N) and per plan for --multiplan (0 = 4096)")
    ap.add_argument("--reps", type=int, default=3, help="timed launches for --rollout-only")
    ap.add_argument("--refit-only", action="store_true",
                    help="time only the select + refit kernel on the move-and-push and pick-place workloads, "
                         "with their initial class mix and with every sample in class 0 (profiling driver)")
    ap.add_argument("--tpr", type=int, default=1,
                    help="lanes per pick-and-place rollout for --rollout-only (1, 8 or 32)")
    ap.add_argument("--controller", choices=["pd", "astar"], default="pd",
                    help="moveTo controller of the pick-place base for --rollout-only pickplace")
    ap.add_argument("--block", type=int, default=0,
                    help="rollout threads per CTA for --rollout-only (0 = the library's choice)")
    ap.add_argument("--skip-surrogate", action="store_true", help="leave out the time-to-cost comparison")
    ap.add_argument("--paper-ce", type=int, default=0,
                    help="run the paper's CE variant on the ramp and box pick-place scenes over this many "
                         "seeds and print the per-iteration success-rate and best-cost curves")
    ap.add_argument("--dr-gain", type=int, default=0,
                    help="optimise the move-and-push task with and without domain randomisation on this many "
                         "seeds and score both plans under fresh randomised environments")
    ap.add_argument("--multiplan", type=int, default=0,
                    help="multi-plan search on this many pick-place scenes (four candidate plans each): "
                         "every plan to the end vs successive halving")
    ap.add_argument("--mlp-only", type=int, default=0,
                    help="time only the surrogate forward on this many rows (profiling driver)")
    ap.add_argument("--batch-only", type=int, default=0,
                    help="time only CE iterations of the first P problems of the 64-problem batch, fixed launch "
                         "shape (--warps, --ctas, --tpr), no graph (profiling driver)")
    ap.add_argument("--warps", type=int, default=4, help="warps per CTA of the persistent launch for --batch-only")
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM of the persistent launch for --batch-only (0 = resident maximum)")
    ap.add_argument("--train-only", type=int, default=0,
                    help="time this many surrogate training steps (batch 4096) on each GEMM path (profiling driver)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def workload_desc(sc, sk, cm):
    return (f"{cm['name']}: N={cm['N']} T={sc['T']} D={len(sk['lo'])} K={cm['K']} dt={sc['dt']} "
            f"(one CE iteration per step, initial distribution)")


def batch_problems(seed, rank):
    """The 64-problem batch with this rank's Philox problem ids."""
    probs = workload.batch_problems(seed)
    for i, p in enumerate(probs):
        p["seed"] = seed
        p["problem"] = 1000 * rank + i
    return probs


def batch_desc(probs, seed):
    steps = sum(p["N"] * p["scene"]["T"] for p in probs)
    by_len = {}
    for p in probs:
        by_len[p["L"]] = by_len.get(p["L"], 0) + 1
    return (f"batched-64: {len(probs)} CE problems (workload.batch_problems(seed={seed})), skeletons of 1..6 "
            f"actions (problems per length {dict(sorted(by_len.items()))}), N per problem in "
            f"[{min(p['N'] for p in probs)}, {max(p['N'] for p in probs)}], T = 400 / 1000 / 3000, "
            f"K = max(8, N/20), full covariance; {steps} simulated steps per CE iteration; "
            f"one step = one CE iteration of every problem (iterations 0..K-1 of one run)")


def batch_flops(probs, seed):
    """Algorithmic flops of one batch iteration: sum over problems of
    flops/step x N x T, from the oracle's counts (per problem for the batch
    the counts were taken on, else the mean per skeleton length)."""
    with open(os.path.join(ROOT, "workload", "flops_per_step.json")) as f:
        tab = json.load(f)["batch-64"]
    per = tab["problems"]
    exact = tab["seed"] == seed and len(probs) <= len(per) and all(
        q["L"] == p["L"] and q["N"] == p["N"] for q, p in zip(per, probs))
    tot = 0.0
    for i, p in enumerate(probs):
        fps = per[i]["flops"] if exact else tab["flops_by_length"][str(p["L"])]
        tot += fps * p["N"] * p["scene"]["T"]
    return tot, ("per problem" if exact else "per skeleton length")


def aggregate(value_units: float, seconds: float, world: int):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([seconds], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
        u = torch.tensor([value_units], dtype=torch.float64, device=t.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        return float(u.item()), float(t.item())
    return value_units, seconds


def flops_per_step(name):
    with open(os.path.join(ROOT, "workload", "flops_per_step.json")) as f:
        return json.load(f)[name]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_batch_iteration(oracle, probs, it, frac, cores):
    """One CE iteration of the FP64 oracle, as it stands, over every problem
    of the batch on a bounded sample: ceil(N / frac) samples per problem
    drawn from its initial distribution at Philox iteration `it`, rolled
    out on `cores` threads, then select + refit with K scaled alike.
    Returns the simulated steps."""
    steps = 0
    for p in probs:
        sc, sk = p["scene"], p["skel"]
        lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
        n = -(-p["N"] // frac)
        th = oracle.sample(p["seed"], it, p["problem"], n, (lo + hi) / 2, np.diag((hi - lo) / 4))
        J, cls = oracle.rollout(sc, sk, th, nthreads=cores)
        idx = oracle.select(J.astype(np.float32), cls, max(1, -(-p["K"] // frac)))
        if len(idx):
            oracle.refit(th, idx, lo, hi)
        steps += n * sc["T"]
    return steps


def cpu_baseline(probs, seconds=10.0, max_iters=50):
    """The FP64 oracle on this host's cores on the same 64-problem batch:
    CE iterations on 1 / CPU_FRACTION of every problem's samples until
    ~`seconds` have passed."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    it, steps, t0 = 0, 0, time.perf_counter()
    while it < max_iters and (time.perf_counter() - t0 < seconds or it == 0):
        steps += oracle_batch_iteration(oracle, probs, it, CPU_FRACTION, cores)
        it += 1
    el = time.perf_counter() - t0
    # one thread: a slice of the largest pick-place problem
    big = max((p for p in probs if p["L"] >= 3), key=lambda p: p["N"])
    lo, hi = np.array(big["skel"]["lo"]), np.array(big["skel"]["hi"])
    n1 = 64
    th = oracle.sample(big["seed"], 0, big["problem"], n1, (lo + hi) / 2, np.diag((hi - lo) / 4))
    t1 = time.perf_counter()
    oracle.rollout(big["scene"], big["skel"], th, nthreads=1)
    el1 = time.perf_counter() - t1
    T1 = big["scene"]["T"]
    return {"value": steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{it} CE iterations of the 64-problem batch on 1/{CPU_FRACTION} of every problem's "
                      f"samples ({steps // max(it, 1)} simulated steps per iteration), FP64, "
                      f"{cores} threads, {el:.1f} s",
            "single_thread": {"value": n1 * T1 / el1, "unit": UNIT,
                              "sample": f"rollouts of {n1} samples of a {big['L']}-action pick-place problem "
                                        f"(T={T1}), 1 thread, {el1:.2f} s"},
            "cpu_model": cpu_model()}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def run_reference(args):
    """The oracle (the reference is a paper without code) on the same
    64-problem batch: each step is one CE iteration of every problem on
    1 / REF_FRACTION of its samples, on this host's cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    probs = batch_problems(args.seed, 0)
    cores = os.cpu_count() or 1
    for j in range(args.warmup):
        oracle_batch_iteration(oracle, probs, j, REF_FRACTION, cores)
    t0 = time.perf_counter()
    steps = 0
    for j in range(args.steps):
        steps += oracle_batch_iteration(oracle, probs, args.warmup + j, REF_FRACTION, cores)
    el = time.perf_counter() - t0
    v = steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": batch_desc(probs, args.seed), "l2": "n/a (host)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"1/{REF_FRACTION} of every problem's samples per CE iteration "
                                   f"({steps // max(args.steps, 1)} simulated steps per step), FP64, "
                                   f"{cores} threads"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_headline(P, args, rank, world, local):
    """The headline: CE iterations of the 64-problem batch, one graph replay
    per step, the L2 flushed (untimed) before each, device-timed with CUDA
    events on the launching stream; the library's own stage events give the
    persistent rollout kernel's time for the roofline.  Then the same run
    end to end through the public API with the state on the host: each step
    restores the state from host memory, iterates once and reads it back."""
    import torch

    probs = batch_problems(args.seed, rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    out = {}
    with P.Batch(probs) as B:
        warps, ctas, best = B.autotune()
        tpr = B.launch()[2]
        B.set_timing(True)
        B.reset(stream)
        B.iterate(args.warmup, use_graph=True, stream=stream)  # capture + warm-up
        torch.cuda.synchronize()
        B.reset(stream)  # the timed steps are iterations 0..K-1 of one run
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        stages = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            t0 = time.perf_counter()
            for j in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(j))  # evict the previous step's data from L2 (untimed)
                evs[j][0].record(stream)
                B.iterate(1, use_graph=True, stream=stream)
                evs[j][1].record(stream)
                stages.append(B.stage_ms())  # waits for this step
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        res = B.read(stream)
        step_ms = [e[0].elapsed_time(e[1]) for e in evs]
        steps_per_iter = B.steps_per_iteration
        # end to end: the CE state crosses the PCIe/C2C link every step
        B.set_timing(False)
        B.reset(stream)
        host = B.read_raw(stream)
        nbytes = B.state_bytes
        B.iterate(1, use_graph=True, stream=stream)  # re-capture without timing events
        torch.cuda.synchronize()
        B.reset(stream)
        host = B.read_raw(stream)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for j in range(args.steps):
            B.set_state(host, stream)
            B.iterate(1, use_graph=True, stream=stream)
            host = B.read_raw(stream)
        e2e_s = time.perf_counter() - t0
        e2e_same = all(int(host[i].best_class) == int(res[i]["best_cls"]) and float(host[i].best_J) == float(res[i]["best_J"])
                       for i in range(len(probs)))
    units, secs = aggregate(steps_per_iter * args.steps, sum(step_ms) / 1e3, world)
    e_units, e_secs = aggregate(steps_per_iter * args.steps, e2e_s, world)
    out.update(probs=probs, steps_per_iter=steps_per_iter, step_ms=step_ms, stages=stages, wall=wall,
               clocks=clk.summary() if rank == 0 else None, value=units / secs,
               e2e=e_units / e_secs, e2e_bytes=nbytes, e2e_same_result=e2e_same,
               launch={"warps_per_cta": warps, "ctas_per_sm": ctas, "lanes_per_pickplace_rollout": tpr,
                       "autotune_best_ms": best},
               classes=np.bincount([r["best_cls"] for r in res], minlength=5).tolist())
    return out


def single_problem(P, cfg, args, rank, steps):
    """One CE iteration from the initial distribution per step on a
    single-problem workload (sample -> rollout -> refit through the C ABI,
    CUDA events around each call, L2 flushed before each step)."""
    import torch

    sc, sk, cm = workload.config(cfg, seed=args.seed)
    N, K, T, D = cm["N"], cm["K"], sc["T"], len(sk["lo"])
    lo, hi = np.array(sk["lo"], np.float32), np.array(sk["hi"], np.float32)
    mean0 = torch.tensor((lo + hi) / 2, device="cuda")
    chol0 = torch.diag(torch.tensor((hi - lo) / 4, device="cuda"))
    cov0 = torch.diag(torch.tensor(((hi - lo) / 4) ** 2, device="cuda"))
    stream = torch.cuda.Stream()
    theta = torch.empty((N, D), device="cuda")
    J = torch.empty(N, device="cuda")
    cls = torch.empty(N, dtype=torch.uint8, device="cuda")
    mean, cov, chol = mean0.clone(), cov0.clone(), chol0.clone()
    idx = torch.empty(K, dtype=torch.int32, device="cuda")
    keff = torch.empty(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with P.Scene(sc, sk) as S:
        def step(j, ev=None):
            with torch.cuda.stream(stream):
                mean.copy_(mean0)
                cov.copy_(cov0)
                chol.copy_(chol0)
                if ev:
                    ev[0].record(stream)
                P.cem_sample(S.h, mean, chol, args.seed, j, rank, N, theta, stream)
                if ev:
                    ev[1].record(stream)
                P.cem_rollout_batch(S.h, theta, N, J, cls, stream)
                if ev:
                    ev[2].record(stream)
                P.cem_refit(S.h, theta, J, cls, N, K, 0, mean, cov, chol, idx, keff, stream)
                if ev:
                    ev[3].record(stream)

        for j in range(3):
            step(j)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        for j in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(j))
            step(3 + j, evs[j])
        torch.cuda.synchronize()
        block, tpr = S.launch(N)
    step_ms = float(np.mean([e[0].elapsed_time(e[3]) for e in evs]))
    roll_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    fps = flops_per_step(cm["name"])["flops"]
    return {"workload": workload_desc(sc, sk, cm), "ms_per_iteration": step_ms,
            "sim_steps_per_s": N * T / (step_ms / 1e3), "rollout_ms": roll_ms,
            "sample_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in evs])),
            "refit_ms": float(np.mean([e[2].elapsed_time(e[3]) for e in evs])),
            "rollout_tflops": fps * N * T / (roll_ms / 1e3) / 1e12, "flops_per_step": fps,
            "launch": {"block": block, "lanes_per_rollout": tpr}, "steps": steps}


def time_to_cost(seed, n_scenes=6):
    """CE time-to-cost, surrogate-screened vs plain, on the pick-place task,
    every CE run one batch of the held-out scenes timed per iteration: a
    surrogate trained on 2,097,152 simulator rollouts (64 training scenes,
    8192 samples each from the initial distribution and after 4, 8 and 16 CE
    iterations), then plain CE (N = 16384, K = 512, 25 iterations), screened
    CE with the same 16384 rollouts per iteration (8192 unscreened + the
    8192 best-scored of the rest of a pool of 65,536) and the literal
    setting (pool 65,536, the 8192 best-scored simulated, K = 512)."""
    import time as _t

    from paper_2512_11571_gb300 import screening

    t0 = _t.perf_counter()
    X, t = screening.training_set(n_scenes=64, per_dist=8192)
    n_rollouts = int(X.shape[0])
    t_data = _t.perf_counter() - t0
    t0 = _t.perf_counter()
    sur, hist = screening.train_surrogate(X, t, steps=3000)
    t_train = _t.perf_counter() - t0
    del X, t
    rows, per_iter = screening.compare_batched(sur, list(range(seed, seed + n_scenes)))
    sur.close()

    def mean(key):
        return float(np.mean([r[key] for r in rows]))

    def faster(name):
        return sum(1 for r in rows if r[f"{name}_ttc_ms"] is not None and r["plain_ttc_ms"] is not None
                   and r[f"{name}_ttc_ms"] < r["plain_ttc_ms"])

    saved = [r["plain_ttc_ms"] - r["screened_ttc_ms"] for r in rows
             if r["screened_ttc_ms"] is not None and r["plain_ttc_ms"] is not None]
    return {"training_rollouts": n_rollouts, "data_s": t_data, "train_s": t_train,
            "train_loss_first_last": [float(hist[:10].mean()), float(hist[-10:].mean())],
            "batched": "each run one batch of the held-out scenes; per-iteration CUDA events",
            "ms_per_iteration": per_iter, "scenes": rows,
            "mean_J": {name: mean(f"{name}_J") for name in ("plain", "screened", "literal")},
            "scenes_faster_than_plain": {name: faster(name) for name in ("screened", "literal")},
            "amortisation": {"surrogate_cost_s": t_data + t_train,
                             "mean_ms_saved_per_scene_run": float(np.mean(saved)) if saved else None,
                             "scene_runs_to_repay": (t_data + t_train) * 1e3 / float(np.mean(saved))
                             if saved and np.mean(saved) > 0 else None}}


def run_gb300(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    hd = batch_headline(P, args, rank, world, local)
    probs = hd["probs"]

    # the single-problem workloads beside it (move-and-push N = 4096,
    # pick-place N = 16384), and the move-and-push rollout with the GPU full
    push = single_problem(P, 1, args, rank, steps=10)
    pick = single_problem(P, 2, args, rank, steps=5)
    sc, sk, cm = workload.config(1, seed=args.seed)
    lo, hi = np.array(sk["lo"], np.float32), np.array(sk["hi"], np.float32)
    D, T = len(sk["lo"]), sc["T"]
    with P.Scene(sc, sk) as S:
        mean0 = torch.tensor((lo + hi) / 2, device="cuda")
        chol0 = torch.diag(torch.tensor((hi - lo) / 4, device="cuda"))
        th_sat = torch.empty((SATURATED_N, D), device="cuda")
        J_sat = torch.empty(SATURATED_N, device="cuda")
        c_sat = torch.empty(SATURATED_N, dtype=torch.uint8, device="cuda")
        st = torch.cuda.current_stream()
        P.cem_sample(S.h, mean0, chol0, args.seed, 0, rank, SATURATED_N, th_sat, st)
        P.cem_rollout_batch(S.h, th_sat, SATURATED_N, J_sat, c_sat, st)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(3):
            P.cem_rollout_batch(S.h, th_sat, SATURATED_N, J_sat, c_sat, st)
        e1.record(st)
        torch.cuda.synchronize()
        sat_ms = e0.elapsed_time(e1) / 3

    # the surrogate forward timed alone (burst peak), before the time-to-cost runs' training
    # and data generation heat the GPU up
    sur = surrogate_roofline(P, args.seed) if rank == 0 and not args.skip_surrogate else None
    # CE time-to-cost: surrogate-screened vs plain (pick-place)
    ttc = time_to_cost(args.seed) if rank == 0 and not args.skip_surrogate else None

    if rank == 0:
        peaks, src = measured_peaks()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        flops, basis = batch_flops(probs, args.seed)
        roll = [s[1] for s in hd["stages"]]
        roll_avg = sum(roll) / len(roll)
        achieved = flops / (roll_avg / 1e3) / 1e12
        ms = sum(hd["step_ms"]) / len(hd["step_ms"])
        fps_push = push["flops_per_step"]
        line = {
            "metric": METRIC, "value": hd["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": batch_desc(probs, args.seed), "problems": len(probs),
                       "sim_steps_per_iteration": hd["steps_per_iter"],
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "sample_ms": float(np.mean([s[0] for s in hd["stages"]])), "rollout_ms": roll_avg,
                       "refit_ms": float(np.mean([s[2] for s in hd["stages"]])), "wall_s": hd["wall"],
                       "launch": hd["launch"], "graph": "one CUDA graph replay per CE iteration",
                       "final_best_class_counts": hd["classes"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "algorithmic_bytes": int(sum(p["N"] * (len(p["skel"]["lo"]) * 4 + 5) for p in probs)),
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {mhz} MHz ({src} max SM clock)",
                         "kernel": "rollout_persistent_kernel",
                         "flops_per_iteration": flops, "flops_basis": f"oracle op counts, {basis}",
                         "timing": "library stage events on the launching stream, every timed step"},
            "e2e": {"value": hd["e2e"], "unit": UNIT, "h2d_bytes_per_step": hd["e2e_bytes"],
                    "d2h_bytes_per_step": hd["e2e_bytes"], "api": "cem_batch_set_state -> cem_batch_iterate -> "
                    "cem_batch_read each step, state in host memory", "same_result_as_device_run": hd["e2e_same_result"]},
            "move_push_N4096": push,
            "pickplace_N16384": pick,
            "roofline_saturated": {"workload": "move-push rollout kernel alone, N = 196,608", "N": SATURATED_N,
                                   "rollout_ms": sat_ms, "sim_steps_per_s": SATURATED_N * T / (sat_ms / 1e3),
                                   "achieved": fps_push * SATURATED_N * T / (sat_ms / 1e3) / 1e12,
                                   "frac": fps_push * SATURATED_N * T / (sat_ms / 1e3) / 1e12 / peak,
                                   "unit": "TFLOP/s"},
            "time_to_cost": ttc,
            "roofline_surrogate": sur,
            "gpu_launches": 5 * args.steps,  # sample, sample order, dispatch order, persistent rollout, refit
            "clocks": hd["clocks"],
        }
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(probs)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_rollout_only(args):
    """Times one workload's rollout kernel alone: one untimed launch, then
    `reps` launches between CUDA events.  Prints one JSON line."""
    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    cfg = {"reach": 0, "push": 1, "pickplace": 2}[args.rollout_only]
    kw = {"controller": args.controller} if cfg == 2 else {}
    sc, sk, cm = workload.config(cfg, seed=args.seed, **kw)
    N = args.n or cm["N"]
    T, D = sc["T"], len(sk["lo"])
    lo, hi = np.array(sk["lo"], np.float32), np.array(sk["hi"], np.float32)
    with P.Scene(sc, sk) as S:
        if args.block:
            P.cem_set_launch(S.h, args.block)
        S.set_threads_per_rollout(args.tpr)
        mean = torch.tensor((lo + hi) / 2, device="cuda")
        chol = torch.tensor(np.diag((hi - lo) / 4), device="cuda")
        theta = S.sample(mean, chol, args.seed, 0, N)
        J, cls = S.rollout(theta)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        for _ in range(args.reps):
            P.cem_rollout_batch(S.h, theta, N, J, cls, st)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
    fps = flops_per_step(cm["name"])
    peaks, _ = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    tf = fps["flops"] * N * T / (ms / 1e3) / 1e12
    print(json.dumps({"rollout_only": cm["name"], "N": N, "T": T, "D": D, "block": args.block, "tpr": args.tpr, "controller": args.controller if cfg == 2 else None, "ms": ms,
                      "sim_steps_per_s": N * T / (ms / 1e3), "achieved_tflops": tf, "frac": tf / peak,
                      "classes": np.bincount(cls.cpu().numpy(), minlength=4).tolist()}), flush=True)


def run_refit_only(args):
    """Times cem_refit alone (20 launches between CUDA events, best of 5) on
    the initial samples of the move-and-push and pick-place workloads: with
    their own classes (few goal samples: K_eff < K, no radix select) and
    with every sample in class 0 (the radix select of the K-th key runs).
    Prints one JSON line with the times and a hash of the elite indices,
    mean, covariance and factor of each case."""
    import hashlib

    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    out = {"refit_only": True}
    for cfg in (1, 2):
        sc, sk, cm = workload.config(cfg, seed=args.seed)
        N, K = cm["N"], cm["K"]
        lo, hi = np.array(sk["lo"], np.float32), np.array(sk["hi"], np.float32)
        with P.Scene(sc, sk) as S:
            m0 = torch.tensor((lo + hi) / 2, device="cuda")
            c0 = torch.tensor(np.diag((hi - lo) / 4), device="cuda")
            th = S.sample(m0, c0, args.seed, 0, N)
            J, cls = S.rollout(th)
            idx = torch.empty(K, dtype=torch.int32, device="cuda")
            ke = torch.empty(1, dtype=torch.int32, device="cuda")
            for name, cc in (("initial", cls), ("all_class0", torch.zeros_like(cls))):
                mean, chol = m0.clone(), c0.clone()
                cov = chol @ chol.T
                P.cem_refit(S.h, th, J, cc, N, K, 0, mean, cov, chol, idx, ke)
                torch.cuda.synchronize()
                best = float("inf")
                for _ in range(5):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(20):
                        P.cem_refit(S.h, th, J, cc, N, K, 0, mean, cov, chol, idx, ke)
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1) / 20 * 1e3)
                k = int(ke.item())
                blob = b"".join(t.cpu().numpy().tobytes() for t in (idx[:k], mean, cov, chol))
                out[f"{cm['name']}/{name}"] = {"N": N, "K": K, "k_eff": k, "us": round(best, 2),
                                               "hash": hashlib.sha256(blob).hexdigest()[:12]}
    print(json.dumps(out), flush=True)


def time_forward_flushed(P, S, x, y, reps):
    """Device time of `reps` surrogate forwards, each after an untimed L2
    flush (the 12.6 MB of features would otherwise stay in the 129 MB L2) and
    between its own CUDA events on the launching stream: (mean, median) ms."""
    import torch

    st = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for j in range(reps):
        flush.fill_(float(j))
        ev[j][0].record(st)
        P.cem_surrogate_forward(S.h, x, y, st)
        ev[j][1].record(st)
    torch.cuda.synchronize()
    t = np.array([a.elapsed_time(b) for a, b in ev])
    return float(t.mean()), float(np.median(t))


def surrogate_roofline(P, seed, M=65536, reps=50, warm=5):
    """The fused tcgen05 surrogate forward (48 -> 4 x 256 GELU -> 1, BF16
    operands, FP32 accumulation) on M rows: `warm` untimed calls, then `reps`
    calls, each after an untimed L2 flush and between its own CUDA events on
    the launching stream; `achieved` uses the mean.  Dense BF16 contraction,
    so the roofline is the measured BF16 tensor peak."""
    import torch

    x = torch.rand((M, 48), device="cuda", generator=torch.Generator("cuda").manual_seed(seed)) * 2 - 1
    flops = 2.0 * M * (48 * 256 + 3 * 256 * 256 + 256)
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    with P.Surrogate(256, 4, seed=seed) as S:
        S.set_forward_path(2)
        y = S.forward(x)
        for _ in range(warm):
            P.cem_surrogate_forward(S.h, x, y, torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms, med = time_forward_flushed(P, S, x, y, reps)
        if S.status() != 0:
            raise SystemExit("surrogate forward: a bounded pipeline wait expired")
    tf = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "mlp_forward_tc_kernel", "rows": M, "ms": ms, "ms_median": med,
            "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "peak_basis": f"bf16_tflops ({src}, burst)", "launches": reps,
            "l2": "flushed before each timed call (256 MiB write, untimed)"}


def run_batch_only(args):
    """CE iterations of the first --batch-only problems of the 64-problem
    batch with a fixed persistent launch shape: --warmup iterations, then
    --steps iterations each timed by the library's stage events.  Prints one
    JSON line with the persistent rollout's time and FP32 fraction."""
    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    probs = batch_problems(args.seed, 0)[:args.batch_only]
    with P.Batch(probs) as B:
        B.set_threads_per_rollout(args.tpr)
        B.set_launch(args.warps, args.ctas)
        B.set_timing(True)
        B.reset()
        B.iterate(args.warmup, use_graph=False)
        roll = []
        for _ in range(args.steps):
            B.iterate(1, use_graph=False)
            roll.append(B.stage_ms()[1])
        torch.cuda.synchronize()
        launch = B.launch()
        steps = B.steps_per_iteration
    peaks, src = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    flops, basis = batch_flops(probs, args.seed)
    ms = float(np.mean(roll))
    tf = flops / (ms / 1e3) / 1e12
    print(json.dumps({"batch_only": len(probs), "sim_steps_per_iteration": steps, "rollout_ms": ms,
                      "rollout_ms_all": roll, "sim_steps_per_s": steps / (ms / 1e3), "achieved_tflops": tf,
                      "frac": tf / peak, "launch": launch, "flops_basis": basis}), flush=True)


def run_train_only(args):
    """Times --train-only AdamW steps of the surrogate (48 -> 4 x 256 -> 1,
    batch 4096 drawn from 65,536 stored rows) with the dense layers on the
    tiled mma.sync GEMM and on the tcgen05 GEMM: 5 untimed steps, then the
    timed ones (each cem_surrogate_train call ends with a device sync)."""
    import numpy as np
    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    rng = np.random.default_rng(args.seed)
    x = torch.tensor(rng.uniform(-1, 1, (65536, 48)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.uniform(0, 1, 65536).astype(np.float32), device="cuda")
    B = 4096
    # forward: 4 layers; backward: weight gradients of 4 layers, input gradients of 3
    gemm_flops = 2.0 * B * ((48 * 256 + 3 * 256 * 256) * 2 + 3 * 256 * 256)
    out = {"train_only": args.train_only, "batch": B, "gemm_gflop_per_step": gemm_flops / 1e9}
    for path, name in ((1, "tiled_mma_sync"), (2, "tcgen05")):
        with P.Surrogate(256, 4, seed=args.seed) as S:
            S.set_gemm_path(path)
            S.train(x, t, batch=B, steps=5, seed=1)
            t0 = time.perf_counter()
            S.train(x, t, batch=B, steps=args.train_only, seed=1)
            ms = (time.perf_counter() - t0) / args.train_only * 1e3
            if S.status() != 0:
                raise SystemExit("surrogate training: a bounded pipeline wait expired")
        out[name] = {"ms_per_step": ms}
    print(json.dumps(out), flush=True)


def run_mlp_only(args):
    """Times the surrogate's BF16 tensor-core forward (4 x 256-wide layers) on
    --mlp-only rows through both paths (the tiled mma.sync GEMM and the fused
    tcgen05 kernel): four untimed calls each, then `reps` calls, each after an
    untimed L2 flush and between its own events."""
    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    M = args.mlp_only
    x = torch.rand((M, 48), device="cuda") * 2 - 1
    flops = 2.0 * M * (48 * 256 + 3 * 256 * 256 + 256)
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    out = {"mlp_only": M, "peak_bf16_tflops": peak, "peak_source": src}
    with P.Surrogate(256, 4, seed=args.seed) as S:
        for path, name in ((1, "tiled_mma_sync"), (2, "fused_tcgen05")):
            S.set_forward_path(path)
            y = S.forward(x)
            for _ in range(3):
                P.cem_surrogate_forward(S.h, x, y, torch.cuda.current_stream())
            torch.cuda.synchronize()
            ms, med = time_forward_flushed(P, S, x, y, args.reps)
            tf = flops / (ms / 1e3) / 1e12
            out[name] = {"ms": ms, "ms_median": med, "tflops": tf, "frac_of_bf16": tf / peak,
                         "l2": "flushed before each timed call"}
        if S.status() != 0:
            raise SystemExit("surrogate forward: a bounded pipeline wait expired")
    print(json.dumps(out), flush=True)


def run_paper_ce(args):
    """The paper's CE variant (uniform start in annulus / box regions, n_env
    3000 -> 300 by iteration 10, N_e = 50, independent normal, 20
    iterations) on the pick-place ramp and box scenes, one scene seed per
    run: per-iteration success rate (class-0 share of the samples, Fig. 5),
    the median best cost so far, and the loop's device time."""
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    out = {"paper_ce": {"n0": 3000, "n1": 300, "j1": 10, "K": 50, "iters": 20, "cov": "diag",
                        "seeds": args.paper_ce}}
    for obstacle in ("ramp", "box"):
        rates, best, ms, cls = [], [], [], []
        for seed in range(args.paper_ce):
            sc, sk = workload.pickplace_scene(seed, obstacle=obstacle, regions="paper")
            with P.Scene(sc, sk) as S:
                r = S.solve_paper(seed)
            rates.append(r["class_counts"][:, 0] / r["n_env"])
            best.append(np.where(np.isfinite(r["history"]), r["history"], np.nan))
            ms.append(r["elapsed_ms"])
            cls.append(int(r["best_cls"]))
        rates, best = np.array(rates), np.array(best)
        out[obstacle] = {
            "success_rate_mean": np.round(rates.mean(0), 5).tolist(),
            "best_J_median": np.round(np.nanmedian(best, 0), 4).tolist(),
            "final_best_class": cls,
            "loop_ms_mean": float(np.mean(ms)),
            "samples_per_loop": int(sum(3000 - 270 * min(j, 10) for j in range(20))),
        }
    print(json.dumps(out), flush=True)


def run_dr_gain(args):
    """Domain randomisation (friction and block mass within +-30 %, 8
    environments per sample) against plain CE on the move-and-push workload
    (N = 4096, K = 200, 20 iterations): each best plan is scored in 8 blocks
    of 32 fresh environments (other Philox seeds) -- the share of blocks in
    which it reaches the goal in every environment, and its mean cost -- and
    one CE iteration of each is timed."""
    import torch

    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    dmu = dm = 0.3
    rows = []
    for seed in range(args.dr_gain):
        sc, sk = workload.push_scene(seed)
        res = {}
        with P.Scene(sc, sk) as S:
            for name, M in (("plain", 1), ("randomised", 8)):
                S.set_randomization(M, dmu if M > 1 else 0.0, dm if M > 1 else 0.0, seed=seed + 1)
                r = S.solve(seed, 4096, 200, 20)
                th = torch.tensor(np.tile(r["best_theta"], (1, 1)), dtype=torch.float32, device="cuda")
                ok, cost = [], []
                for b in range(8):
                    S.set_randomization(32, dmu, dm, seed=10_000 + 97 * seed + b)
                    J, cls = S.rollout(th)
                    ok.append(int(cls.item()) == 0)
                    cost.append(float(J.item()))
                res[name] = {"robust_success": float(np.mean(ok)), "mean_cost": float(np.mean(cost)),
                             "ms_per_iteration": r["elapsed_ms"] / 20, "best_cls": int(r["best_cls"])}
        rows.append(res)
    out = {"dr_gain": {"task": "move-and-push", "N": 4096, "K": 200, "iters": 20, "M": 8,
                       "delta_mu": dmu, "delta_mass": dm, "eval_blocks": 8, "eval_envs_per_block": 32}}
    for name in ("plain", "randomised"):
        out[name] = {k: float(np.mean([r[name][k] for r in rows])) for k in rows[0][name]}
        out[name]["per_seed_robust_success"] = [r[name]["robust_success"] for r in rows]
    print(json.dumps(out), flush=True)


def run_multiplan(args):
    """Four candidate plans per pick-place scene (direct, and three 6-action
    plans through waypoints) realised in one batch, N = 4096, K = 200, 20
    iterations: every plan for all iterations vs successive halving every 5
    iterations.  Reports the chosen plan and cost of both, the simulated
    steps and the wall time (host clock around the synchronous call)."""
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    rows = []
    N = args.n or 4096
    for seed in range(args.multiplan):
        sc, plans = workload.pickplace_plans(seed)
        row = {}
        for name, halving in (("all_plans", 0), ("halving", 5)):
            P.cem_multiplan_solve(sc, plans, seed=seed, N=N, K=200, iters=1)  # warm-up
            t0 = time.perf_counter()
            res, best = P.cem_multiplan_solve(sc, plans, seed=seed, N=N, K=200, iters=20, halving_iters=halving)
            ms = (time.perf_counter() - t0) * 1e3
            row[name] = {"best_plan": best, "best_J": float(res[best]["best_J"]), "best_cls": int(res[best]["best_cls"]),
                         "iters_per_plan": [r["iters_run"] for r in res],
                         "sim_steps": int(sum(r["iters_run"] for r in res) * N * sc["T"]), "ms": ms}
        rows.append(row)
    out = {"multiplan": {"plans": 4, "N": N, "K": 200, "iters": 20, "halving_iters": 5, "scenes": rows}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.multiplan:
        run_multiplan(args)
        return
    if args.dr_gain:
        run_dr_gain(args)
        return
    if args.paper_ce:
        run_paper_ce(args)
        return
    if args.train_only:
        run_train_only(args)
        return
    if args.batch_only:
        run_batch_only(args)
        return
    if args.mlp_only:
        run_mlp_only(args)
        return
    if args.rollout_only:
        run_rollout_only(args)
        return
    if args.refit_only:
        run_refit_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
