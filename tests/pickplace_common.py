"""Shared set-up of the pick-and-place tests: a converged CE distribution
per scene from the FP64 oracle's own CE (N = 512, K = 50, 10 iterations of
Algorithm 1), after which most samples finish all five actions of the plan
(move, grasp, move, place, move to the exit), so grasp, carry, place and
release are all exercised.  Test infrastructure: the distribution comes
from the oracle only."""
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
