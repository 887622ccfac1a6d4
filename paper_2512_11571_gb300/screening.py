"""Surrogate-screened CE on the pick-place task: training data from the
simulator, training, and the screened-vs-plain comparison.

Sequencing only: every sample, rollout, feature, target, training step and
screening step runs in libcemtamp's kernels; torch holds device memory.

Training data: for each training scene, equal numbers of samples from the
initial CE distribution and from the distributions after 4, 8 and 16 plain
CE iterations on that scene (the regions CE visits later, where screening
has to tell good candidates apart); target = log(1 + J + 10 * class).  Screening keeps CE's simulation budget and elite
rule (elites from simulated costs only) and spends the surrogate on choosing
which candidates of a larger pool get simulated, keeping an unscreened
exploration share so that the elite set is not confined to the surrogate's
predicted basin.
"""
from __future__ import annotations

import numpy as np

import workload

from . import COV, Batch, Scene, Surrogate, cem_surrogate_targets  # noqa: F401


def _dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def training_set(n_scenes=64, per_dist=8192, stages=(4, 8, 16), seed0=10 ** 6, surrogate=None, streams=8):
    """(X [n_scenes * per_dist * (len(stages) + 1), 48], t) on the device from
    pick-place scenes seed0 .. seed0 + n_scenes - 1: per scene, per_dist
    samples from the initial distribution and from the CE distribution after
    each stage's iteration count.  The CE of all scenes runs as one batch
    (one persistent rollout launch per iteration); the scenes' sample
    rollouts then run on `streams` CUDA streams at once, so the GPU is full
    although one scene's rollouts alone would leave most SMs idle."""
    import torch

    own = surrogate is None
    sur = Surrogate(64, 1) if own else surrogate
    specs = []
    for s in range(n_scenes):
        sc, sk, _ = workload.config(2, seed=seed0 + s)
        specs.append((sc, sk, workload.scene_features(sc), np.array(sk["lo"]), np.array(sk["hi"])))
    probs = [dict(scene=sc, skel=sk, N=4096, K=256, seed=s, problem=s) for s, (sc, sk, *_) in enumerate(specs)]
    dists = [[(_dev((lo + hi) / 2), _dev(np.diag((hi - lo) / 4)))] for (_, _, _, lo, hi) in specs]
    with Batch(probs) as B:
        done = 0
        for st in stages:
            B.iterate(st - done)
            done = st
            for s, r in enumerate(B.read()):
                dists[s].append((_dev(r["mean"]), _dev(r["chol"])))
    scenes = [Scene(sc, sk) for sc, sk, *_ in specs]
    X, T = [], []
    try:
        torch.cuda.synchronize()  # inputs in place before other streams read them
        pool = [torch.cuda.Stream() for _ in range(streams)]
        out = []
        for s, S in enumerate(scenes):
            with torch.cuda.stream(pool[s % streams]):
                for j, (m, c) in enumerate(dists[s]):
                    th = S.sample(m, c, 77 + s, j, per_dist)
                    J, cls = S.rollout(th)
                    t = torch.empty_like(J)
                    cem_surrogate_targets(J, cls, t)
                    out.append((s, th, t))
        torch.cuda.synchronize()
        # features one scene after another (the surrogate context holds one scene's tables)
        for s, th, t in out:
            _, _, f16, lo, hi = specs[s]
            X.append(sur.features(th, lo, hi, f16))
            T.append(t)
        x, tt = torch.cat(X), torch.cat(T)
        torch.cuda.synchronize()
    finally:
        for S in scenes:
            S.close()
        if own:
            sur.close()
    return x, tt


def training_set_serial(n_scenes=64, per_dist=8192, stages=(4, 8, 16), seed0=10 ** 6, surrogate=None):
    """training_set one scene at a time (cem_solve for each scene's CE, every
    launch on the current stream): the reference for the batched version."""
    import torch

    own = surrogate is None
    sur = Surrogate(64, 1) if own else surrogate
    X, T = [], []
    try:
        for s in range(n_scenes):
            sc, sk, _ = workload.config(2, seed=seed0 + s)
            f16 = workload.scene_features(sc)
            lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
            with Scene(sc, sk) as S:
                dists = [((lo + hi) / 2, np.diag((hi - lo) / 4))]
                for st in stages:
                    r = S.solve(s, 4096, 256, st)
                    dists.append((r["mean"], r["chol"]))
                for j, (m, c) in enumerate(dists):
                    th = S.sample(_dev(m), _dev(c), 77 + s, j, per_dist)
                    J, cls = S.rollout(th)
                    t = torch.empty_like(J)
                    cem_surrogate_targets(J, cls, t)
                    X.append(sur.features(th, lo, hi, f16))
                    T.append(t)
    finally:
        if own:
            sur.close()
    return torch.cat(X), torch.cat(T)


def train_surrogate(X, t, width=256, depth=4, steps=3000, batch=8192, lr=1e-3, seed=0):
    sur = Surrogate(width, depth, seed=seed)
    hist = sur.train(X, t, batch=batch, steps=steps, lr=lr, weight_decay=1e-4, seed=seed + 1)
    return sur, hist


def compare(sur, scene_seeds, N=16384, K=512, iters=25, n_pool=65536, n_explore=8192, finetune=None):
    """Plain CE and surrogate-screened CE (same rollouts per iteration) on
    held-out scenes: final best cost, loop time, and time to reach 1% of the
    plain run's final cost.  finetune (a dict for Scene.solve_screened): also
    a screened run whose surrogate fine-tunes on the run's own samples; every
    screened run starts from the surrogate as given, which is restored at the
    end."""
    w0, n0 = sur.params()
    rows = []
    for s in scene_seeds:
        sc, sk, _ = workload.config(2, seed=s)
        f16 = workload.scene_features(sc)
        c = None
        with Scene(sc, sk) as S:
            S.solve(s, N, K, 1)  # warm-up (allocation, graph)
            a = S.solve(s, N, K, iters)
            sur.set_params(w0, n0)
            b = S.solve_screened(sur, f16, seed=s, N=N, K=K, iters=iters, n_pool=n_pool, n_explore=n_explore)
            if finetune is not None:
                sur.set_params(w0, n0)
                c = S.solve_screened(sur, f16, seed=s, N=N, K=K, iters=iters, n_pool=n_pool, n_explore=n_explore,
                                     finetune=dict(finetune, seed=s))
        target = 1.01 * a["best_J"]

        def ttc(r):
            t = r["elapsed_ms"] * np.arange(1, iters + 1) / iters
            ok = np.where(r["history"] <= target)[0]
            return float(t[ok[0]]) if len(ok) else None

        row = dict(scene=s, plain_J=float(a["best_J"]), plain_ms=a["elapsed_ms"], plain_cls=a["best_cls"],
                   screened_J=float(b["best_J"]), screened_ms=b["elapsed_ms"], screened_cls=b["best_cls"],
                   plain_ttc_ms=ttc(a), screened_ttc_ms=ttc(b))
        if c is not None:  # loop time includes the fine-tuning steps
            row.update(finetuned_J=float(c["best_J"]), finetuned_ms=c["elapsed_ms"], finetuned_cls=c["best_cls"])
        rows.append(row)
    sur.set_params(w0, n0)
    return rows


def _batched_run(specs, sur, N, K, iters, n_pool=0, n_explore=0):
    """One CE run of every held-out scene as one batch (plain when sur is
    None, else screened): device time of each iteration (CUDA events on the
    launching stream around it) and every scene's best cost after it."""
    import torch

    probs = [dict(scene=sc, skel=sk, N=N, K=K, seed=s, problem=s) for s, sc, sk, _ in specs]
    f16 = np.stack([f for *_, f in specs])
    st = torch.cuda.current_stream()
    with Batch(probs) as B:
        if sur is not None:
            B.set_screening(sur, f16, n_pool, n_explore)
        step = (lambda: B.iterate_screened(1, st)) if sur is not None else (lambda: B.iterate(1, True, st))
        step()  # warm-up (workspaces, graph capture), then a fresh run
        B.reset()
        ms, best = [], []
        for _ in range(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            step()
            e1.record(st)
            res = B.read()  # synchronises
            ms.append(e0.elapsed_time(e1))
            best.append([(r["best_cls"], float(r["best_J"])) for r in res])
        if sur is not None and sur.status() != 0:
            raise RuntimeError("surrogate forward: a bounded pipeline wait expired")
    return np.array(ms), best


def compare_batched(sur, scene_seeds, N=16384, K=512, iters=25, n_pool=65536, n_explore=8192, n_literal=8192):
    """Plain CE and surrogate-screened CE on held-out pick-place scenes, each
    run as ONE batch of all the scenes, timed per iteration with CUDA events:
      plain     -- N = 16384 rollouts per scene and iteration;
      screened  -- the same N rollouts: n_explore unscreened draws and the
                   best-scored N - n_explore of the rest of a pool of n_pool;
      literal   -- a pool of n_pool, the n_literal best-scored simulated
                   (no unscreened draws), K elites from simulated costs.
    Per scene: final best cost of each run, and the device time each run
    takes to first reach the plain run's final cost within 1%."""
    specs = []
    for s in scene_seeds:
        sc, sk, _ = workload.config(2, seed=s)
        specs.append((s, sc, sk, workload.scene_features(sc)))
    runs = {"plain": _batched_run(specs, None, N, K, iters),
            "screened": _batched_run(specs, sur, N, K, iters, n_pool, n_explore),
            "literal": _batched_run(specs, sur, n_literal, K, iters, n_pool, 0)}
    rows = []
    for i, (s, *_rest) in enumerate(specs):
        plain_cls, plain_J = runs["plain"][1][-1][i]
        target = 1.01 * plain_J
        row = dict(scene=s, plain_J=plain_J, plain_cls=plain_cls)
        for name, (ms, best) in runs.items():
            cum = np.cumsum(ms)
            hit = [j for j in range(iters) if best[j][i][0] <= plain_cls and best[j][i][1] <= target]
            row[f"{name}_J"] = best[-1][i][1]
            row[f"{name}_cls"] = best[-1][i][0]
            row[f"{name}_ttc_ms"] = float(cum[hit[0]]) if hit else None
        rows.append(row)
    per_iter = {name: float(np.mean(ms)) for name, (ms, _) in runs.items()}
    return rows, per_iter
