"""What the trained surrogate gains: surrogate-screened CE against plain CE
(and against the same screening with an untrained network) on held-out
pick-place scenes, with the same rollouts per iteration.  The pipeline is
deterministic (Philox sampling, fixed-order reductions), so the outcome is a
fixed property of the code, not a random draw."""
import numpy as np
import pytest

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


def test_trained_surrogate_improves_screened_ce(P):
    from paper_2512_11571_gb300 import screening

    X, t = screening.training_set(n_scenes=32, per_dist=8192)
    assert X.shape == (32 * 4 * 8192, 48)
    sur, hist = screening.train_surrogate(X, t, steps=2000)
    # the training set now includes late-stage CE samples, whose costs sit
    # close together relative to the target normalisation: a larger share of
    # the normalised loss is irreducible, so the bar is a two-thirds drop
    assert hist[-50:].mean() < 0.35 * hist[:5].mean()
    scenes = list(range(6))
    trained = screening.compare(sur, scenes)
    untrained_net = P.Surrogate(256, 4, seed=99)
    untrained = screening.compare(untrained_net, scenes)
    sur.close()
    untrained_net.close()
    pj = np.array([r["plain_J"] for r in trained])
    sj = np.array([r["screened_J"] for r in trained])
    uj = np.array([r["screened_J"] for r in untrained])
    print("plain", pj.round(4), "screened", sj.round(4), "untrained-screened", uj.round(4))
    # the trained network beats the same screening with random scores, and
    # the screened loop is no worse than plain CE on average
    assert sj.mean() < uj.mean()
    assert sj.mean() <= pj.mean() * 1.005
