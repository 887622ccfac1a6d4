"""Shared set-up of the pick-and-place tests: a converged CE distribution
per scene from the FP64 oracle's own CE (N = 512, K = 50, 10 iterations of
Algorithm 1), after which most samples finish all five actions of the plan
(move, grasp, move, place, move to the exit), so grasp, carry, place and
release are all exercised.  Test infrastructure: the distribution comes
from the oracle only.  Also the comparison helpers the pick-and-place
parity tests share: the borderline probe, the per-step state bar and the
action-transition steps."""
import functools

import numpy as np

import workload

# trace columns (the per-step state layout of a pick-place rollout)
BX, BY, OX, OY, OZ, OVX, OVY, OVZ, ATT, ACT, EX, EY, EZ = 0, 1, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19
GRIP = 4  # theta index of the grasp's grip-height offset
SEEDS = (0, 1, 5)


@functools.lru_cache(maxsize=None)
def converged(seed):
    """(scene, skeleton, mean, Cholesky factor) after the oracle's CE."""
    import oracle

    oracle.build()
    sc, sk, _ = workload.config(2, seed=seed)
    r = oracle.cem(sc, sk, seed=seed, N=512, K=50, iters=10)
    return sc, sk, r["mean"], np.linalg.cholesky(r["cov"])


def events(tr):
    """(attach step, release step) of one trace, None where there is none."""
    att = tr[:, ATT]
    on = np.where(np.diff(att) > 0.5)[0]
    off = np.where(np.diff(att) < -0.5)[0]
    return (int(on[0]) + 1 if len(on) else None), (int(off[0]) + 1 if len(off) else None)


def borderline(roll, sk, th, J0, idx, tol=1e-3, reps=8, seed=0, radius=1e-6):
    """For each sample in idx: does its FP64 cost move by more than tol
    (relative) when theta moves by `radius` of its range in one of `reps`
    random directions?  Such a sample sits within rounding of a discrete
    event (a success test, a contact onset, a waypoint switch, the object
    sliding off a table edge).  roll(thetas) is the oracle's cost of a stack
    of parameter vectors."""
    rng = np.random.default_rng(seed)
    span = np.array(sk["hi"]) - np.array(sk["lo"])
    out = []
    for i in idx:
        thp = []
        for _ in range(reps):
            u = rng.standard_normal(len(span))
            thp.append(th[i].astype(np.float64) + radius * span * u / np.linalg.norm(u))
        Jp = roll(np.array(thp))
        out.append(bool(np.any(np.abs(Jp - J0[i]) / max(abs(J0[i]), 1e-3) > tol)))
    return np.array(out, bool)


def nearby_outcome(roll, sk, th, idx, J, cls, tol=1e-3, radii=(1e-6, 1e-5), reps=16, seed=0):
    """For each sample in idx: is the device's (cost, class) the FP64
    outcome of a nearby parameter vector, theta moved by one of `radii` of
    its range in one of `reps` random directions (cost within tol relative,
    class equal)?  Near a discrete event the FP32 trajectory can take the
    branch that a perturbation of this size takes; this accepts exactly
    that, and nothing the FP64 model cannot produce close by.
    roll(thetas) -> (costs, classes) of the oracle."""
    rng = np.random.default_rng(seed)
    span = np.array(sk["hi"]) - np.array(sk["lo"])
    out = []
    for i in idx:
        thp = []
        for r in radii:
            for _ in range(reps):
                u = rng.standard_normal(len(span))
                thp.append(th[i].astype(np.float64) + r * span * u / np.linalg.norm(u))
        Jp, cp = roll(np.array(thp))
        out.append(bool(np.any((np.abs(Jp - J[i]) <= tol * np.maximum(np.abs(Jp), 1e-3)) & (cp == cls[i]))))
    return np.array(out, bool)


# Per-step state bar over the grasp -> carry -> place -> release segment.
# Each FP32 step rounds every state variable by ~6e-8 |x|; the PD laws and
# friction clamps damp these errors with time constants of ~100 steps, so
# they settle near a few 1e-6 m (measured: positions <= 2.3e-6 m, angles
# <= 2.3e-6 rad, velocities <= 7e-5 m/s over 3 scenes x 64 samples).  The
# bar is 1e-4 m / 1e-4 rad for positions and angles and 1e-3 m/s / rad/s
# for velocities: some 40x above that error scale and 500x below the
# success tolerance eps = 0.05 m that decides every action's end, so a
# sequencing slip of the kind the oracle's pins target (an offset, a release
# velocity, a wrong step) is far outside it.  The azimuth is compared modulo
# 2 pi; the attachment flag and the action index exactly.
POS_COLS = (0, 1, 4, 5, 9, 10, 11, 17, 18, 19)
VEL_COLS = (2, 3, 6, 7, 12, 13, 14)


def state_error(gpu, ref):
    """(worst ratio to the bar, its (step, column)) of one trace segment."""
    d = np.abs(gpu - ref)
    d[:, 8] = np.abs((gpu[:, 8] - ref[:, 8] + np.pi) % (2 * np.pi) - np.pi)
    bar = np.full(d.shape[1], np.inf)
    bar[list(POS_COLS) + [8]] = 1e-4
    bar[list(VEL_COLS)] = 1e-3
    ratio = d / bar
    ratio[:, [ATT, ACT]] = np.where(d[:, [ATT, ACT]] == 0.0, 0.0, np.inf)
    i = np.unravel_index(np.argmax(ratio), ratio.shape)
    return float(ratio[i]), i


def transitions(tr):
    """Step at which each action index is first reached."""
    a = tr[:, ACT].astype(int)
    return {int(k): int(np.argmax(a >= k)) for k in range(1, a.max() + 1)}
