"""Out-of-memory paths through the C ABI, by host-side fault injection.

cem_test_fail_allocation(k) makes the k-th next device allocation of the
library report cudaErrorMemoryAllocation without allocating (no GPU memory
is exhausted, nothing faults).  For every call that allocates -- scene
creation, the solve workspace, batch creation, the surrogate and its
screening pool, the A* path query -- the test fails its 1st, 2nd, ...
allocation in turn until the call goes through: each failure returns
CEM_ERR_NO_MEMORY, hands out no handle, leaves the device's free memory
where it was (what the call had allocated is released), and the call then
gives the result of a run that never failed."""
import numpy as np
import pytest

import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ALLOCS = 64  # more than any one call makes


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    return P


def free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # blocks the binding's own tensors left in torch's cache
    return torch.cuda.mem_get_info()[0]


def fail_each_allocation(P, call):
    """Run call() with its k-th allocation failing, k = 1, 2, ... until it
    succeeds; returns (its result, the number of failures seen)."""
    for k in range(1, MAX_ALLOCS + 1):
        before = free_bytes()
        P.cem_test_fail_allocation(k)
        try:
            out = call()
        except P.CemError as e:
            assert P.STATUS[e.code] == "CEM_ERR_NO_MEMORY", (k, str(e))
            assert free_bytes() == before, (k, "device memory leaked on the failure path")
            continue
        finally:
            P.cem_test_fail_allocation(0)
        return out, k - 1
    raise AssertionError("the call kept allocating")


def solve_once(P, sc, sk):
    with P.Scene(sc, sk) as S:
        return S.solve(5, 512, 32, 2, problem=1, use_graph=False)


def same(a, b):
    assert a["best_cls"] == b["best_cls"] and a["best_J"] == b["best_J"]
    assert np.array_equal(a["best_theta"], b["best_theta"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["cov"], b["cov"])


def test_scene_and_solve_workspace(P):
    sc, sk = workload.pickplace_scene(2, T=300)
    ref = solve_once(P, sc, sk)  # also loads every kernel the calls below use
    out, n = fail_each_allocation(P, lambda: solve_once(P, sc, sk))
    assert n >= 5  # the scene, then the solve workspace's four device arrays
    same(out, ref)


def test_batch_creation(P):
    probs = []
    for i, (sc, sk) in enumerate([workload.reach_scene(0), workload.push_scene(1, T=300),
                                  workload.pickplace_scene(3, T=300)]):
        probs.append(dict(scene=sc, skel=sk, N=100 + 37 * i, K=8, seed=i, problem=i))

    def run():
        with P.Batch(probs) as B:
            B.iterate(2, use_graph=False)
            return B.read()

    ref = run()
    out, n = fail_each_allocation(P, run)
    assert n >= 10
    for a, b in zip(out, ref):
        same(a, b)


def test_surrogate_and_screening_pool(P):
    sc, sk, _ = workload.config(2, seed=3)
    f16 = workload.scene_features(sc)

    def run():
        with P.Scene(sc, sk, T=300) as Sc, P.Surrogate(256, 4, seed=4) as S:
            return Sc.solve_screened(S, f16, seed=1, N=256, K=16, iters=2, n_pool=2048)

    ref = run()
    out, n = fail_each_allocation(P, run)
    assert n >= 8
    same(out, ref)


def test_base_path_buffers(P):
    sc, sk = workload.pickplace_scene(0, controller="astar")
    with P.Scene(sc, sk) as S:
        start, goal = tuple(sc["base_start"][:2]), tuple(sk["actions"][0]["nominal"][:2])
        ref = S.base_path(start, goal)
        out, n = fail_each_allocation(P, lambda: S.base_path(start, goal))
    assert n == 2 and np.array_equal(out, ref)  # the waypoint buffer, then the count


def test_hook_validation_and_reset(P):
    with pytest.raises(P.CemError):
        P.cem_test_fail_allocation(-1)
    P.cem_test_fail_allocation(1000)  # armed far ahead, then switched off: nothing fails
    P.cem_test_fail_allocation(0)
    sc, sk = workload.reach_scene(0)
    assert np.isfinite(solve_once(P, sc, sk)["best_J"])
