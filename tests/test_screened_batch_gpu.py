"""Batched surrogate-screened CE through the C ABI: every problem of a
screened batch equals the single-problem screened loop (cem_solve_screened)
of that problem bit for bit -- the same pool draws, scores, kept candidates,
rollouts and refits -- whatever the surrogate's forward path; bad settings
are refused."""
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


def scenes(n=3, T=900):
    out = []
    for i in range(n):
        sc, sk = workload.pickplace_scene(200 + i, T=T)
        out.append((sc, sk, workload.scene_features(sc)))
    return out


@pytest.mark.parametrize("width,depth", [(256, 4), (64, 2)])
def test_screened_batch_equals_single_screened_solves(P, width, depth):
    N, K, n_pool, n_explore, iters = 1000, 64, 4096, 200, 3
    sc3 = scenes()
    probs = [dict(scene=sc, skel=sk, N=N, K=K, seed=7 + i, problem=40 + i) for i, (sc, sk, _) in enumerate(sc3)]
    f16 = np.stack([f for _, _, f in sc3])
    with P.Surrogate(width, depth, seed=3) as S:
        with P.Batch(probs) as B:
            B.set_screening(S, f16, n_pool, n_explore)
            B.iterate_screened(iters)
            got = B.read()
        assert S.status() == 0
        for i, (sc, sk, f) in enumerate(sc3):
            with P.Scene(sc, sk) as Sc:
                ref = Sc.solve_screened(S, f, seed=7 + i, N=N, K=K, iters=iters, n_pool=n_pool, n_explore=n_explore,
                                        problem=40 + i)
            g = got[i]
            assert g["best_cls"] == ref["best_cls"] and g["best_J"] == ref["best_J"]
            assert np.array_equal(g["best_theta"], ref["best_theta"])
            assert np.array_equal(g["mean"], ref["mean"]) and np.array_equal(g["cov"], ref["cov"])
            assert g["iters_done"] == iters


def test_screening_settings_are_checked(P):
    sc3 = scenes(2, T=200)
    probs = [dict(scene=sc, skel=sk, N=512, K=32, seed=i) for i, (sc, sk, _) in enumerate(sc3)]
    f16 = np.stack([f for _, _, f in sc3])
    with P.Surrogate(64, 2) as S, P.Batch(probs) as B:
        with pytest.raises(P.CemError):
            B.iterate_screened(1)  # no surrogate set yet
        with pytest.raises(P.CemError):
            B.set_screening(S, f16, 256, 0)  # pool smaller than N
        with pytest.raises(P.CemError):
            B.set_screening(S, f16, 4096, 600)  # more unscreened draws than N
        with pytest.raises(ValueError):
            B.set_screening(S, f16[:1], 4096, 0)  # one scene row per problem
        B.set_screening(S, f16, 4096, 100)
        B.iterate_screened(1)
        B.set_screening(None, None, 0)
        with pytest.raises(P.CemError):
            B.iterate_screened(1)
        B.iterate(1)  # plain iterations still run
        r = B.read()
        assert all(x["iters_done"] == 2 for x in r)
