"""Benchmark of the CE plan-realization hot path on GB300.

One step = one cross-entropy iteration of Algorithm 1 on the move-and-push
workload (N = 4096 samples, T = 1000 steps, D = 6, K = 200): Philox sample ->
fused rollout -> elite select + refit, all on the device through the C ABI.
Reported value: simulated steps per second (N x T / time per iteration).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs an independent replica (its own Philox
problem id) on its own GPU: weak scaling, no data-path collective.
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
CONFIG = 1  # the move-and-push workload
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SATURATED_N = 48 * 4096  # enough rollouts to give every SM scheduler several warps
# DRAM bytes (read + write) of one rollout launch of this workload from the
# ncu capture in profiles/rollout_push_N4096_T1000.md; reported only while the
# kernel source still matches the one the counters were taken on
ROLLOUT_TRAFFIC = {"rollout.cu sha256[:16]": "6c45f86787854617", "bytes": 127232}


def rollout_traffic():
    import hashlib

    path = os.path.join(ROOT, "paper_2512_11571_gb300", "csrc", "rollout.cu")
    with open(path, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return ROLLOUT_TRAFFIC["bytes"] if h == ROLLOUT_TRAFFIC["rollout.cu sha256[:16]"] else None


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


def cpu_baseline(sc, sk, cm, seconds=10.0, max_reps=20):
    """The FP64 oracle, as it stands, on this host's cores: full CE
    iterations of the same workload until ~`seconds` have passed."""
    import oracle

    oracle.build()
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    mean, chol = (lo + hi) / 2, np.diag((hi - lo) / 4)
    cores = os.cpu_count() or 1
    N, T = cm["N"], sc["T"]
    reps, t0 = 0, time.perf_counter()
    while reps < max_reps and (time.perf_counter() - t0 < seconds or reps == 0):
        th = oracle.sample(1, reps, 0, N, mean, chol)
        J, cls = oracle.rollout(sc, sk, th, nthreads=cores)
        idx = oracle.select(J.astype(np.float32), cls, cm["K"])
        oracle.refit(th, idx, lo, hi)
        reps += 1
    el = time.perf_counter() - t0
    # one thread: rollouts of a bounded slice of the same batch
    n1 = min(N, 1024)
    th = oracle.sample(1, 0, 0, n1, mean, chol)
    t1 = time.perf_counter()
    oracle.rollout(sc, sk, th, nthreads=1)
    el1 = time.perf_counter() - t1
    return {"value": reps * N * T / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} full CE iterations (N={N}, T={T}) of the same workload, FP64, "
                      f"{cores} threads, {el:.1f} s",
            "single_thread": {"value": n1 * T / el1, "unit": UNIT,
                              "sample": f"rollouts of {n1} samples (T={T}), 1 thread, {el1:.2f} s"},
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
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc, sk, cm = workload.config(CONFIG, seed=args.seed)
    import oracle

    oracle.build()
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    mean, chol = (lo + hi) / 2, np.diag((hi - lo) / 4)
    cores = os.cpu_count() or 1
    n_sample = 512  # bounded sample of the N = 4096 batch per step
    T = sc["T"]

    def step(j):
        th = oracle.sample(1, j, 0, n_sample, mean, chol)
        J, cls = oracle.rollout(sc, sk, th, nthreads=cores)
        idx = oracle.select(J.astype(np.float32), cls, min(cm["K"], n_sample))
        oracle.refit(th, idx, lo, hi)

    for j in range(args.warmup):
        step(j)
    t0 = time.perf_counter()
    for j in range(args.steps):
        step(args.warmup + j)
    el = time.perf_counter() - t0
    v = args.steps * n_sample * T / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(sc, sk, cm), "l2": "n/a (host)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_sample} of the {cm['N']} samples per CE iteration, T={T}, FP64"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_measurement(P, seed, rank, iters=3):
    """64 independent problems (skeletons of 1..6 actions, uneven N and T)
    advanced together: CE iterations per second and simulated steps per
    second of the whole batch, launch shape chosen by the autotuner."""
    import torch

    probs = workload.batch_problems(seed)
    for i, p in enumerate(probs):
        p["seed"] = seed
        p["problem"] = 1000 * rank + i
    with P.Batch(probs) as B:
        warps, ctas, _ = B.autotune()
        B.reset()
        B.iterate(1, use_graph=True)  # capture + warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        B.iterate(iters, use_graph=True, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        steps = B.steps_per_iteration
    return {"problems": len(probs), "sim_steps_per_iteration": steps, "ms_per_iteration": ms,
            "sim_steps_per_s": steps / (ms / 1e3), "launch": {"warps_per_cta": warps, "ctas_per_sm": ctas},
            "kernels_per_iteration": 3}


def time_to_cost(seed):
    """CE time-to-cost, surrogate-screened vs plain, on the pick-place task:
    a surrogate trained on 2,097,152 simulator rollouts (64 training scenes,
    8192 samples each from the initial distribution and after 4, 8 and 16 CE
    iterations),
    then plain CE (N = 16384, K = 512, 25 iterations) and screened CE (pool
    65536, the same 16384 rollouts per iteration, 8192 of them unscreened)
    on three held-out scenes; a third run fine-tunes the surrogate on its own
    samples (100 AdamW steps of 4096 after every 5 iterations, replay ring of
    65,536)."""
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
    ft = dict(every=5, steps=100, batch=4096, capacity=65536, lr=5e-4, weight_decay=1e-4)
    rows = screening.compare(sur, [seed, seed + 1, seed + 2], finetune=ft)
    sur.close()
    return {"training_rollouts": n_rollouts, "data_s": t_data, "train_s": t_train,
            "train_loss_first_last": [float(hist[:10].mean()), float(hist[-10:].mean())], "scenes": rows,
            "mean_plain_J": float(np.mean([r["plain_J"] for r in rows])),
            "mean_screened_J": float(np.mean([r["screened_J"] for r in rows])),
            "finetune": ft, "mean_finetuned_J": float(np.mean([r["finetuned_J"] for r in rows]))}


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
    sc, sk, cm = workload.config(CONFIG, seed=args.seed)
    N, K, T, D = cm["N"], cm["K"], sc["T"], len(sk["lo"])
    lo, hi = np.array(sk["lo"], np.float32), np.array(sk["hi"], np.float32)
    mean0 = torch.tensor((lo + hi) / 2, device="cuda")
    chol0 = torch.tensor(np.diag((hi - lo) / 4), device="cuda")
    cov0 = chol0 @ chol0.T
    S = P.Scene(sc, sk)
    stream = torch.cuda.Stream()
    theta = torch.empty((N, D), device="cuda")
    J = torch.empty(N, device="cuda")
    cls = torch.empty(N, dtype=torch.uint8, device="cuda")
    mean, cov, chol = mean0.clone(), cov0.clone(), chol0.clone()
    idx = torch.empty(K, dtype=torch.int32, device="cuda")
    keff = torch.empty(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    problem = rank

    def step(j, ev=None):
        # every step: one CE iteration from the initial distribution
        with torch.cuda.stream(stream):
            mean.copy_(mean0)
            cov.copy_(cov0)
            chol.copy_(chol0)
            if ev:
                ev[0].record(stream)
            P.cem_sample(S.h, mean, chol, args.seed, j, problem, N, theta, stream)
            if ev:
                ev[1].record(stream)
            P.cem_rollout_batch(S.h, theta, N, J, cls, stream)
            if ev:
                ev[2].record(stream)
            P.cem_refit(S.h, theta, J, cls, N, K, 0, mean, cov, chol, idx, keff, stream)
            if ev:
                ev[3].record(stream)

    for j in range(args.warmup):
        step(j)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for j in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(j))  # evict the previous step's data from L2 (untimed)
            step(args.warmup + j, evs[j])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    roll_ms = [e[1].elapsed_time(e[2]) for e in evs]
    samp_ms = [e[0].elapsed_time(e[1]) for e in evs]
    refit_ms = [e[2].elapsed_time(e[3]) for e in evs]
    ms = sum(step_ms) / args.steps
    units, secs = aggregate(N * T * args.steps, sum(step_ms) / 1e3, world)
    value = units / secs

    # the same rollout kernel with the GPU full (context for the roofline
    # fraction: N = 4096 leaves most SM schedulers without a warp)
    th_sat = torch.empty((SATURATED_N, D), device="cuda")
    J_sat = torch.empty(SATURATED_N, device="cuda")
    c_sat = torch.empty(SATURATED_N, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        P.cem_sample(S.h, mean0, chol0, args.seed, 0, problem, SATURATED_N, th_sat, stream)
        P.cem_rollout_batch(S.h, th_sat, SATURATED_N, J_sat, c_sat, stream)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            P.cem_rollout_batch(S.h, th_sat, SATURATED_N, J_sat, c_sat, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    sat_ms = e0.elapsed_time(e1) / 3

    # the 64-problem batched workload: one persistent launch per iteration
    batch = batched_measurement(P, args.seed, rank)

    # CE time-to-cost: surrogate-screened vs plain (pick-place)
    ttc = time_to_cost(args.seed) if rank == 0 and not args.skip_surrogate else None
    sur = surrogate_roofline(P, args.seed) if rank == 0 and not args.skip_surrogate else None

    # end to end through the public API with host buffers: cem_solve, one
    # iteration per step, distribution in from pinned host memory and the
    # best sample / new distribution back to the host
    init_mean = np.ascontiguousarray((lo + hi) / 2, np.float32)
    init_cov = np.ascontiguousarray(np.diag(((hi - lo) / 4) ** 2), np.float32)
    S.solve(args.seed, N, K, 1, init_mean=init_mean, init_cov=init_cov)  # allocate + capture
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for j in range(args.steps):
        S.solve(args.seed, N, K, 1, init_mean=init_mean, init_cov=init_cov, start_iter=j)
    e2e_s = time.perf_counter() - t0
    e_units, e_secs = aggregate(N * T * args.steps, e2e_s, world)
    # cem_solve moves its small state as one block each way (capi.cu: loop
    # state 96 B, status, k_eff, mean / cov / chol at the 18-parameter
    # maximum, each 16-byte aligned: 2800 B), plus the 1-iteration histories
    # the binding asks for (best cost, k_eff, class counts)
    h2d = 2800
    d2h = 2800 + 4 + 4 + 16

    if rank == 0:
        fps = flops_per_step(cm["name"])
        peaks, src = measured_peaks()
        clocks = clk.summary()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roll_avg = sum(roll_ms) / len(roll_ms)
        achieved = fps["flops"] * N * T / (roll_avg / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(sc, sk, cm), "N": N, "T": T, "D": D, "K": K,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "rollout_ms": roll_avg, "sample_ms": sum(samp_ms) / len(samp_ms),
                       "refit_ms": sum(refit_ms) / len(refit_ms), "wall_s": wall},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": rollout_traffic(),
                         "algorithmic_bytes": N * D * 4 + N * 5,
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                       f"({src} max SM clock)",
                         "kernel": "rollout_kernel<PUSH>",
                         "flops_per_step": fps["flops"]},
            "roofline_saturated": {"N": SATURATED_N, "rollout_ms": sat_ms,
                                   "sim_steps_per_s": SATURATED_N * T / (sat_ms / 1e3),
                                   "achieved": fps["flops"] * SATURATED_N * T / (sat_ms / 1e3) / 1e12,
                                   "frac": fps["flops"] * SATURATED_N * T / (sat_ms / 1e3) / 1e12 / peak,
                                   "unit": "TFLOP/s"},
            "e2e": {"value": e_units / e_secs, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "batched_64": batch,
            "time_to_cost": ttc,
            "roofline_surrogate": sur,
            "gpu_launches": 3 * args.steps,
            "gpu_launches_outside_timed_region": 5 + 3 * (args.steps + 1),
            "clocks": clocks,
        }
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(sc, sk, cm)
        print(json.dumps(line), flush=True)
    S.close()
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


def surrogate_roofline(P, seed, M=65536, reps=20):
    """The fused tcgen05 surrogate forward (48 -> 4 x 256 GELU -> 1, BF16
    operands, FP32 accumulation) on M rows: one untimed call, then `reps`
    calls between CUDA events on the launching stream.  Dense BF16
    contraction, so the roofline is the measured BF16 tensor peak."""
    import torch

    x = torch.rand((M, 48), device="cuda", generator=torch.Generator("cuda").manual_seed(seed)) * 2 - 1
    flops = 2.0 * M * (48 * 256 + 3 * 256 * 256 + 256)
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    with P.Surrogate(256, 4, seed=seed) as S:
        S.set_forward_path(2)
        y = S.forward(x)
        st = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            P.cem_surrogate_forward(S.h, x, y, st)
        e1.record(st)
        torch.cuda.synchronize()
        if S.status() != 0:
            raise SystemExit("surrogate forward: a bounded pipeline wait expired")
    ms = e0.elapsed_time(e1) / reps
    tf = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "mlp_forward_tc_kernel", "rows": M, "ms": ms, "achieved": tf,
            "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "peak_basis": f"bf16_tflops ({src}, burst)", "launches": reps}


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
    tcgen05 kernel): one untimed call each, then `reps` calls between events."""
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
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st = torch.cuda.current_stream()
            e0.record(st)
            for _ in range(args.reps):
                P.cem_surrogate_forward(S.h, x, y, st)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            tf = flops / (ms / 1e3) / 1e12
            out[name] = {"ms": ms, "tflops": tf, "frac_of_bf16": tf / peak}
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
