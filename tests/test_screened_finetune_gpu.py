"""Online fine-tuning of the surrogate inside the screened CE loop.

With fine-tuning switched off the loop equals cem_solve_screened bit for
bit (the replay ring only records); switched on, the surrogate's weights
move, the CE state stays valid (elites from simulated costs only) and the
run is deterministic; bad fine-tune parameters are rejected."""
import numpy as np
import pytest

import workload
from oracle import mlp

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


def surrogate(P):
    S = P.Surrogate(256, 4, seed=1)
    S.set_params(mlp.flatten(mlp.init_params(48, 256, 4, seed=2)), np.array([1.0, 0.5]))
    return S


def run(P, finetune, N=1024, iters=6):
    sc, sk, _ = workload.config(2, seed=3, T=600)
    f16 = workload.scene_features(sc)
    with surrogate(P) as Sg, P.Scene(sc, sk) as S:
        r = S.solve_screened(Sg, f16, seed=5, N=N, K=64, iters=iters, n_pool=4 * N, n_explore=N // 2,
                             finetune=finetune)
        w = Sg.params()[0]
    return r, w


def test_finetune_off_equals_plain_screened(P):
    a, wa = run(P, None)
    b, wb = run(P, dict(every=0, capacity=4096))
    assert a["best_J"] == b["best_J"] and a["best_cls"] == b["best_cls"]
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["history"], b["history"])
    assert np.array_equal(wa, wb)


def test_finetune_updates_weights_deterministically(P):
    ft = dict(every=2, steps=20, batch=512, capacity=2048, lr=1e-3, seed=7)
    a, wa = run(P, ft)
    b, wb = run(P, ft)
    _, w0 = run(P, None)
    assert not np.array_equal(wa, w0)  # the surrogate learned from the run
    assert np.array_equal(wa, wb) and a["best_J"] == b["best_J"]
    assert np.isfinite(a["best_J"]) and a["iters_done"] == 6
    assert np.all(np.diff(a["history"]) <= 0)  # best-ever cost never rises


@pytest.mark.parametrize("bad", [dict(capacity=1000), dict(capacity=0), dict(every=-1), dict(batch=0),
                                 dict(steps=-5)])
def test_finetune_validation(P, bad):
    ft = dict(every=2, steps=10, batch=256, capacity=2048)
    ft.update(bad)
    with pytest.raises(P.CemError):
        run(P, ft, iters=2)
