"""The surrogate's training GEMMs on tcgen05 against the tiled mma.sync path
and the FP64 oracle.

Both paths form the same BF16 products with FP32 accumulation (in a
different order), so their gradients agree to BF16 tolerance, and each
matches the exact FP64 chain rule as in the plain gradient test.  The shapes
cover both operand majors (the weight-gradient GEMMs read both operands
transposed, the input-gradient GEMMs one), split-K over a ragged batch,
N = 48 (the first layer's weight gradient), hidden widths 64 / 128 / 256,
and batches that leave a ragged last row tile."""
import numpy as np
import pytest

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


def layer_blocks(g, grads):
    o = 0
    for (gW, gb) in grads:
        for ref in (gW.reshape(-1), gb):
            yield g[o:o + ref.size], ref
            o += ref.size


def test_gemm_path_selection(P):
    with P.Surrogate(256, 4) as S:
        assert S.gemm_path == 2  # automatic: tcgen05
        S.set_gemm_path(1)
        assert S.gemm_path == 1
        S.set_gemm_path(2)
        assert S.gemm_path == 2
        S.set_gemm_path(3)  # the FP32 debug gradient
        assert S.gemm_path == 3
        for bad in (-1, 4):
            with pytest.raises(P.CemError):
                S.set_gemm_path(bad)


@pytest.mark.parametrize("M,width,depth", [(256, 256, 4), (3001, 256, 4), (1000, 128, 3), (777, 64, 2)])
def test_gradients_agree_between_paths(P, M, width, depth):
    params = mlp.init_params(48, width, depth, seed=M + width)
    rng = np.random.default_rng(M)
    X = rng.uniform(-1, 1, (M, 48))
    t = np.sin(X[:, 0] * 2) + X[:, 1] * X[:, 2]
    got = {}
    with P.Surrogate(width, depth) as S:
        S.set_params(mlp.flatten(params), np.array([0.0, 1.0]))
        for path in (1, 2):
            S.set_gemm_path(path)
            got[path] = S.gradient(dev(X), dev(t))
        assert S.status() == 0
    loss_ref, grads = mlp.loss_and_grads(params, X, t)
    for path in (1, 2):
        g, loss = got[path]
        assert abs(loss - loss_ref) <= 2e-2 * loss_ref
        for a, ref in layer_blocks(g, grads):
            assert np.linalg.norm(a - ref) <= 3e-2 * np.linalg.norm(ref) + 1e-7
    # the two paths: same products, only the FP32 summation order differs
    (g1, l1), (g2, l2) = got[1], got[2]
    assert abs(l1 - l2) <= 1e-3 * abs(l1)
    for (a, ref), (b, _) in zip(layer_blocks(g1, grads), layer_blocks(g2, grads)):
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(a) + 1e-7


def test_training_agrees_between_paths(P):
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (20000, 48)).astype(np.float32)
    t = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 40]).astype(np.float32)
    hist = {}
    for path in (1, 2):
        with P.Surrogate(256, 4, seed=3) as S:
            S.set_gemm_path(path)
            hist[path] = S.train(dev(X), dev(t), batch=2048, steps=150, lr=2e-3, seed=4)
            assert S.status() == 0
    for path in (1, 2):
        assert hist[path][-10:].mean() < 0.3 * hist[path][:3].mean()
    # the same run up to rounding: early losses nearly equal, final losses close
    np.testing.assert_allclose(hist[1][:3], hist[2][:3], rtol=1e-2)
    assert abs(hist[1][-10:].mean() - hist[2][-10:].mean()) <= 0.15 * hist[1][-10:].mean()


def test_tcgen05_training_is_deterministic(P):
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (5000, 48)).astype(np.float32)
    t = X[:, 3].astype(np.float32)
    out = []
    for _ in range(2):
        with P.Surrogate(128, 2, seed=5) as S:
            S.set_gemm_path(2)
            S.train(dev(X), dev(t), batch=1000, steps=20, seed=1)
            out.append(S.params()[0])
    assert np.array_equal(out[0], out[1])
