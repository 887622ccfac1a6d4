"""Threads per rollout: a group of 8 or 32 lanes shares one pick-and-place
rollout, splitting the per-geometry contact queries and neighbour-list
rebuilds and summing contact forces with warp shuffles in ascending
geometry order.  Every lane width must give bit-identical J and class to
one lane per rollout, in single-problem launches of any block shape, in
the persistent batched launch, and in the CE loops built on them."""
import numpy as np
import pytest

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


def rollouts(P, S, theta, tpr, block):
    S.set_threads_per_rollout(tpr)
    S.set_launch(block)
    J, cls = S.rollout(theta)
    torch.cuda.synchronize()
    return J.cpu().numpy(), cls.cpu().numpy()


# ramp and box obstacles, 3..6 actions; N ragged against every group and block
@pytest.mark.parametrize("seed,L,obstacle,N", [(0, 5, "ramp", 1000), (3, 3, "box", 777), (5, 6, "ramp", 301)])
def test_lane_widths_are_bit_identical(P, seed, L, obstacle, N):
    sc, sk = workload.pickplace_scene(seed, n_actions=L, obstacle=obstacle)
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    with P.Scene(sc, sk) as S:
        mean = torch.tensor((lo + hi) / 2, dtype=torch.float32, device="cuda")
        chol = torch.tensor(np.diag((hi - lo) / 4), dtype=torch.float32, device="cuda")
        theta = S.sample(mean, chol, seed, 0, N)
        J1, c1 = rollouts(P, S, theta, 1, 64)
        for tpr, block in ((1, 2), (1, 4), (1, 8), (1, 16), (8, 32), (8, 256), (32, 32), (32, 128)):
            J, c = rollouts(P, S, theta, tpr, block)
            assert np.array_equal(c, c1), (tpr, block)
            assert np.array_equal(J.view(np.uint32), J1.view(np.uint32)), (tpr, block)
        assert S.launch(N) == (128, 32)
    assert np.all(np.isfinite(J1))


def test_cem_solve_with_lane_groups(P):
    sc, sk, _ = workload.config(2, seed=2, T=800)
    with P.Scene(sc, sk) as S:
        ref = S.solve(4, 512, 32, 3, use_graph=True)
        S.set_threads_per_rollout(8)
        got = S.solve(4, 512, 32, 3, use_graph=True)
        S.set_threads_per_rollout(32)
        got32 = S.solve(4, 512, 32, 3, use_graph=False)
    for g in (got, got32):
        assert g["best_J"] == ref["best_J"] and g["best_cls"] == ref["best_cls"]
        assert np.array_equal(g["mean"], ref["mean"]) and np.array_equal(g["cov"], ref["cov"])


def mixed_problems():
    probs = []
    sc, sk = workload.reach_scene(0)
    probs.append(dict(scene=sc, skel=sk, N=200, K=20, seed=11))
    sc, sk = workload.push_scene(1)
    probs.append(dict(scene=sc, skel=sk, N=333, K=30, seed=12))
    for L in (3, 5, 6):
        sc, sk = workload.pickplace_scene(2 + L, n_actions=L, T=700, obstacle="box" if L == 5 else "ramp")
        probs.append(dict(scene=sc, skel=sk, N=96 + 40 * L, K=16, seed=20 + L))
    for i, p in enumerate(probs):
        p["problem"] = 200 + i
    return probs


@pytest.mark.parametrize("tpr,warps", [(8, 4), (32, 2), (8, 1)])
def test_batch_lane_widths_are_bit_identical(P, tpr, warps):
    probs = mixed_problems()
    with P.Batch(probs) as B:
        B.iterate(3, use_graph=False)
        ref = B.read()
        B.reset()
        B.set_launch(warps, 0)
        B.set_threads_per_rollout(tpr)
        assert B.launch()[0] == warps and B.launch()[2] == tpr
        B.iterate(3, use_graph=True)
        got = B.read()
    for a, b in zip(got, ref):
        assert a["best_J"] == b["best_J"] and a["best_cls"] == b["best_cls"]
        assert np.array_equal(a["best_theta"], b["best_theta"])
        assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["cov"], b["cov"])


def test_autotuners_pick_a_supported_shape(P, tmp_path):
    sc, sk = workload.pickplace_scene(1, T=600)
    cache = str(tmp_path / "tune.txt")
    with P.Scene(sc, sk) as S:
        b = S.autotune(2048, cache)
        block, tpr = S.launch(2048)
        assert block == b and tpr in (1, 8, 32)
    line = open(cache).read().strip().split("|")
    assert int(line[1]) == b and int(line[2]) == tpr
    with P.Scene(sc, sk) as S:  # from the cache
        assert S.autotune(2048, cache) == b and S.launch(2048) == (b, tpr)
    with P.Batch(mixed_problems()) as B:
        B.autotune()
        w, c, t = B.launch()
        assert 1 <= w <= 8 and c >= 1 and t in (1, 8, 32)


def test_lane_width_validation(P):
    sc, sk = workload.push_scene(0)
    with P.Scene(sc, sk) as S:
        for bad in (0, 2, 16, 64):
            with pytest.raises(P.CemError):
                S.set_threads_per_rollout(bad)
        S.set_threads_per_rollout(8)  # accepted; push rollouts keep one lane
        assert S.launch(4096)[1] == 1


def test_default_launch_shapes(P):
    """Pick-and-place with one lane per rollout takes few lanes per CTA when
    N is small (lanes in different actions diverge), the other scenes keep
    16-thread CTAs; an explicit block size wins."""
    sc, sk, _ = workload.config(2, seed=0)
    with P.Scene(sc, sk) as S:
        assert S.launch(4096) == (2, 1)
        assert S.launch(16384) == (8, 1)
        assert S.launch(65536)[0] == 32
        S.set_launch(64)
        assert S.launch(4096) == (64, 1)
    sc, sk, _ = workload.config(1, seed=0)
    with P.Scene(sc, sk) as S:
        assert S.launch(4096) == (16, 1)
