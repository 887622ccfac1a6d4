"""Multi-plan search (one scene, several candidate plans in one persistent
batch, optional successive halving) and the batch's active set.

Every plan advances by the batch kernels exactly as cem_solve advances it,
so each plan's result must equal cem_solve of that plan for the iterations
it ran, bit for bit; the elimination order and the chosen plan must follow
the (class, cost, plan index) ranking of those results.  On a quadratic
cost whose plans differ only in their bounds, the chosen plan must be the
one whose box holds the minimiser, and agree with the oracle's CE."""
import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    return P


def single(P, scene, skel, seed, N, K, iters, problem):
    with P.Scene(scene, skel) as S:
        return S.solve(seed, N, K, iters, problem=problem, use_graph=False)


def same(a, b):
    assert a["best_cls"] == b["best_cls"] and a["best_J"] == b["best_J"]
    assert np.array_equal(a["best_theta"], b["best_theta"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["cov"], b["cov"])


def key(r, i):
    return (r["best_cls"], r["best_J"], i)


def test_every_plan_equals_its_own_solve(P):
    sc, plans = workload.pickplace_plans(1)
    res, best = P.cem_multiplan_solve(sc, plans, seed=5, N=256, K=16, iters=4)
    for i, (r, sk) in enumerate(zip(res, plans)):
        assert r["iters_run"] == 4 and r["iters_done"] == 4
        same(r, single(P, sc, sk, 5, 256, 16, 4, i))
    assert best == min(range(len(res)), key=lambda i: key(res[i], i))


def test_successive_halving_follows_the_ranking(P):
    sc, plans = workload.pickplace_plans(2)
    seed, N, K = 3, 256, 16
    res, best = P.cem_multiplan_solve(sc, plans, seed=seed, N=N, K=K, iters=10, halving_iters=3, keep=1)
    runs = [r["iters_run"] for r in res]
    assert sorted(runs) == [3, 3, 6, 10]  # 4 plans -> 2 after 3 iterations -> 1 after 6
    for i, r in enumerate(res):
        assert r["iters_done"] == runs[i]
        same(r, single(P, sc, plans[i], seed, N, K, runs[i], i))
    # replay the eliminations from single solves
    at3 = [single(P, sc, plans[i], seed, N, K, 3, i) for i in range(4)]
    order3 = sorted(range(4), key=lambda i: key(at3[i], i))
    assert sorted(runs[i] for i in order3[:2]) == [6, 10] and all(runs[i] == 3 for i in order3[2:])
    two = [i for i in range(4) if runs[i] > 3]
    at6 = {i: single(P, sc, plans[i], seed, N, K, 6, i) for i in two}
    win6 = min(two, key=lambda i: key(at6[i], i))
    assert runs[win6] == 10 and best == win6


def quadratic_plans():
    sc, sk = workload.quadratic_scene(2, D=4)
    ts = np.array(sc["theta_star"])
    plans = []
    for shift in (0.9, 0.0, -0.9):  # only the unshifted box holds theta*
        lo = np.clip(ts - 0.4 + shift, -1.0, 1.0)
        hi = np.clip(ts + 0.4 + shift, -1.0, 1.0)
        plans.append(dict(sk, lo=lo.tolist(), hi=hi.tolist()))
    return sc, plans


@pytest.mark.parametrize("halving", [0, 2])
def test_quadratic_plans_choose_the_box_with_the_minimiser(P, halving):
    sc, plans = quadratic_plans()
    res, best = P.cem_multiplan_solve(sc, plans, seed=4, N=512, K=32, iters=8, halving_iters=halving)
    assert best == 1 and res[1]["best_J"] < 1e-3 and res[1]["iters_run"] == 8
    orc = [oracle.cem(sc, sk, 4, 512, 32, 8, problem=i) for i, sk in enumerate(plans)]
    assert min(range(3), key=lambda i: (orc[i]["best_cls"], orc[i]["best_J"], i)) == best
    for i in range(3):
        if res[i]["iters_run"] == 8:
            assert res[i]["best_J"] == pytest.approx(orc[i]["best_J"], rel=1e-3, abs=1e-4)


def test_batch_active_set(P):
    probs = []
    for i in range(4):
        sc, sk = workload.push_scene(i, T=400)
        probs.append(dict(scene=sc, skel=sk, N=300, K=20, seed=9, problem=50 + i))
    with P.Batch(probs) as B:
        B.iterate(2)
        with pytest.raises(ValueError, match="one flag per problem"):
            B.set_active([1, 0, 1])
        with pytest.raises(ValueError, match="holds 4 problems"):
            P.cem_batch_read(B.h, 3)
        B.set_active([1, 0, 1, 0])
        B.iterate(3)
        got = B.read()
        assert [g["iters_done"] for g in got] == [5, 2, 5, 2]
        B.reset()  # everyone active again
        B.iterate(1)
        assert [g["iters_done"] for g in B.read()] == [1, 1, 1, 1]
    for i, pr in enumerate(probs):
        same(got[i], single(P, pr["scene"], pr["skel"], 9, 300, 20, 5 if i % 2 == 0 else 2, 50 + i))
