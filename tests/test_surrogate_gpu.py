"""The BF16 tensor-core surrogate kernels against the FP64 MLP oracle.

Forward: against the oracle with the library's BF16 rounding points
emulated (only FP32-vs-exact accumulation differs) and against plain FP64
(BF16 tolerance).  Gradients: against the exact FP64 chain rule at BF16
tolerance (relative error of each layer's gradient <= 3e-2).  Training:
the loss falls on a smooth target.  Screening: the kept candidates are the
lowest scores with ties broken by index, bit-exact against numpy."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("N", [1, 257, 1000])
def test_targets_match_oracle(P, N):
    """Regression targets of simulated samples (FP32 log1p) against the FP64
    definition, with negative, infinite and NaN costs and every class."""
    rng = np.random.default_rng(N)
    J = rng.uniform(-1.0, 30.0, N).astype(np.float32)
    cls = rng.integers(0, 4, N).astype(np.uint8)
    J[::7] = np.inf
    J[3::11] = np.nan
    t = torch.empty(N, dtype=torch.float32, device="cuda")
    P.cem_surrogate_targets(dev(J), torch.as_tensor(cls).cuda(), t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t.cpu().numpy(), mlp.targets(J, cls), rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("M,width,depth", [(1, 256, 4), (1000, 256, 4), (4097, 64, 2), (300, 200, 3)])
def test_forward_matches_oracle(P, M, width, depth):
    params = mlp.init_params(48, width, depth, seed=M)
    rng = np.random.default_rng(M)
    X = rng.uniform(-1.5, 1.5, (M, 48))
    with P.Surrogate(width, depth) as S:
        S.set_params(mlp.flatten(params), np.array([0.0, 1.0]))
        y = S.forward(dev(X)).cpu().numpy().astype(np.float64)
    ye, _ = mlp.forward(params, X, emulate_bf16=True)
    y64, _ = mlp.forward(params, X)
    scale = max(1.0, np.abs(y64).max())
    assert np.median(np.abs(y - ye)) <= 1e-4 * scale
    assert np.max(np.abs(y - ye)) <= 2e-2 * scale
    assert np.max(np.abs(y - y64)) <= 5e-2 * scale


def test_output_denormalisation(P):
    params = mlp.init_params(48, 64, 2, seed=1)
    X = np.random.default_rng(1).uniform(-1, 1, (100, 48))
    with P.Surrogate(64, 2) as S:
        S.set_params(mlp.flatten(params), np.array([0.0, 1.0]))
        y0 = S.forward(dev(X)).cpu().numpy()
        S.set_params(mlp.flatten(params), np.array([3.0, 2.5]))
        y1 = S.forward(dev(X)).cpu().numpy()
    np.testing.assert_allclose(y1, 3.0 + 2.5 * y0, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("M", [256, 4096, 3001])
def test_gradient_matches_fp64(P, M):
    params = mlp.init_params(48, 256, 4, seed=7)
    rng = np.random.default_rng(M)
    X = rng.uniform(-1, 1, (M, 48))
    t = np.sin(X[:, 0] * 2) + X[:, 1] * X[:, 2]
    with P.Surrogate(256, 4) as S:
        S.set_params(mlp.flatten(params), np.array([0.0, 1.0]))
        g, loss = S.gradient(dev(X), dev(t))
    loss_ref, grads = mlp.loss_and_grads(params, X, t)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    o = 0
    for (gW, gb) in grads:
        for ref in (gW.reshape(-1), gb):
            got = g[o:o + ref.size]
            o += ref.size
            assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref) + 1e-7


def test_training_reduces_loss(P):
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (65536, 48)).astype(np.float32)
    t = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 40] + 10.0).astype(np.float32)
    with P.Surrogate(256, 4, seed=2) as S:
        hist = S.train(dev(X), dev(t), batch=2048, steps=400, lr=2e-3, seed=9)
        _, norm = S.params()
        y = S.forward(dev(X[:4096])).cpu().numpy()
    assert abs(norm[0] - t.mean()) < 1e-3 and abs(norm[1] - t.std()) < 1e-3
    assert hist[-20:].mean() < 0.1 * hist[:5].mean()
    resid = np.sqrt(np.mean((y - t[:4096]) ** 2))
    assert resid < 0.3 * t.std()


def test_training_is_deterministic(P):
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (5000, 48)).astype(np.float32)
    t = X[:, 3].astype(np.float32)
    out = []
    for _ in range(2):
        with P.Surrogate(64, 2, seed=5) as S:
            S.train(dev(X), dev(t), batch=512, steps=30, seed=1)
            out.append(S.params()[0])
    assert np.array_equal(out[0], out[1])


def test_features_match_oracle(P):
    sc, sk, _ = workload.config(2, seed=1)
    f16 = workload.scene_features(sc)
    rng = np.random.default_rng(0)
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    th = rng.uniform(lo - 0.3 * (hi - lo), hi + 0.3 * (hi - lo), (777, len(lo))).astype(np.float32)
    with P.Surrogate(64, 1) as S:
        x = S.features(dev(th), lo, hi, f16).cpu().numpy()
    np.testing.assert_allclose(x, mlp.features(th, lo, hi, f16), rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("n_pool,n_keep", [(65536, 8192), (1000, 999), (777, 777), (5000, 1)])
def test_screen_keeps_lowest_scores(P, n_pool, n_keep):
    sc, sk, _ = workload.config(2, seed=2)
    f16 = workload.scene_features(sc)
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    mean = dev((lo + hi) / 2)
    chol = dev(np.diag((hi - lo) / 4))
    with P.Scene(sc, sk) as Sc, P.Surrogate(64, 2, seed=3) as S:
        keep = torch.empty((n_keep, len(lo)), device="cuda")
        idx = torch.empty(n_keep, dtype=torch.int32, device="cuda")
        P.cem_surrogate_screen(Sc.h, S.h, mean, chol, 5, 2, 1, n_pool, n_keep, f16, keep, idx)
        pool = Sc.sample(mean, chol, 5, 2, n_pool, problem=1)
        score = S.forward(S.features(pool, lo, hi, f16)).cpu().numpy()
        torch.cuda.synchronize()
    order = np.lexsort((np.arange(n_pool), score))[:n_keep]
    expect = np.sort(order)
    assert np.array_equal(idx.cpu().numpy(), expect)
    assert np.array_equal(keep.cpu().numpy(), pool.cpu().numpy()[expect])


def test_screened_solve_runs(P):
    sc, sk, _ = workload.config(2, seed=3)
    f16 = workload.scene_features(sc)
    with P.Scene(sc, sk, T=600) as Sc, P.Surrogate(64, 2, seed=4) as S:
        r = Sc.solve_screened(S, f16, seed=1, N=512, K=32, iters=3, n_pool=4096)
    assert r["iters_done"] == 3 and np.isfinite(r["best_J"]) and r["best_cls"] <= 2


def test_batched_training_set_matches_serial(P):
    """The batched generator (one batch for the warm-up CE, sample rollouts on
    several streams) gives the serial generator's rows for the initial
    distribution bit for bit; the warm-distribution rows come from the same
    procedure under the batch's per-problem random streams."""
    from paper_2512_11571_gb300 import screening

    n, per, stages = 3, 1024, (2, 4)
    Xb, tb = screening.training_set(n_scenes=n, per_dist=per, stages=stages, streams=2)
    Xs, ts = screening.training_set_serial(n_scenes=n, per_dist=per, stages=stages)
    Xb, tb, Xs, ts = (a.cpu().numpy() for a in (Xb, tb, Xs, ts))
    rows_per_scene = per * (len(stages) + 1)
    assert Xb.shape == Xs.shape == (n * rows_per_scene, 48) and tb.shape == ts.shape == (n * rows_per_scene,)
    assert np.all(np.isfinite(Xb)) and np.all(np.isfinite(tb))
    for s in range(n):
        rows = slice(s * rows_per_scene, s * rows_per_scene + per)  # the initial-distribution block of scene s
        assert np.array_equal(Xb[rows], Xs[rows]) and np.array_equal(tb[rows], ts[rows])
