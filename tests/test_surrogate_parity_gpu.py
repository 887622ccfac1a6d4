"""Surrogate training against the FP64 MLP oracle, element by element.

Gradients (mean squared error of the 48 -> 4 x 256 GELU -> 1 network, every
weight and bias tensor):

  * the BF16 training paths (tiled mma.sync and tcgen05) against the
    oracle's BF16-emulating backward, which rounds at the library's storage
    points (inputs, weights, hidden activations, hidden-layer gradients) and
    is exact in between, so only the library's FP32 accumulation and its
    occasional different BF16 rounding of a near-tie differ: every element
    within 1e-2 relative, the denominator max(|g|, rms of the tensor) (an
    element far below the tensor's typical size is a cancellation whose
    error is set by the typical terms), and 1e-3 on each tensor's norm;
  * the FP32 debug path (gemm path 3: FP32 end to end, compensated sums)
    against the exact FP64 chain rule: 1e-6 on each tensor's norm of the
    error relative to its norm, and every element within 1e-4 (the FP32
    GELU and GELU' carry a few units in the last place per element).

AdamW: one step of the library's optimiser kernel against the oracle's
step from the same FP32 state and the same (FP32-valued) constants, at step
1 and at step 1000 (bias correction 1 - beta^t), every element within the
FP32 error of one step (derived term by term in step_error_bound); and
1000 chained steps within the drift that FP32 moments allow.
"""
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


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def problem(M, seed=7):
    """FP32-representable parameters, inputs and targets (both sides start
    from the very same numbers)."""
    params = [(f32(W), f32(b)) for W, b in mlp.init_params(48, 256, 4, seed=seed)]
    rng = np.random.default_rng(M)
    X = f32(rng.uniform(-1, 1, (M, 48)))
    t = f32(np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2])
    return params, X, t


def gpu_gradient(P, params, X, t, path):
    with P.Surrogate(256, 4) as S:
        S.set_params(mlp.flatten(params), np.array([0.0, 1.0]))
        S.set_gemm_path(path)
        assert S.gemm_path == (3 if path == 3 else path)
        g, loss = S.gradient(dev(X), dev(t))
    return g.astype(np.float64), loss


def tensors(flat, ref):
    o = 0
    for l, (gW, gb) in enumerate(ref):
        for name, r in (("W", gW.reshape(-1)), ("b", gb)):
            yield f"{name}{l}", flat[o:o + r.size], r
            o += r.size


@pytest.mark.parametrize("M", [256, 3001, 4096])
@pytest.mark.parametrize("path", [1, 2])
def test_bf16_gradients_element_by_element(P, M, path):
    params, X, t = problem(M)
    g, loss = gpu_gradient(P, params, X, t, path)
    loss_ref, ref = mlp.loss_and_grads(params, X, t, emulate_bf16=True)
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    for name, got, r in tensors(g, ref):
        d = np.abs(got - r)
        rms = np.sqrt(np.mean(r * r))
        worst = (d / np.maximum(np.abs(r), rms)).max()
        assert worst <= 1e-2, (name, worst)
        assert np.linalg.norm(d) <= 1e-3 * np.linalg.norm(r), (name, np.linalg.norm(d) / np.linalg.norm(r))


@pytest.mark.parametrize("M", [256, 3001, 4096])
def test_fp32_debug_gradients_against_exact(P, M):
    params, X, t = problem(M)
    g, loss = gpu_gradient(P, params, X, t, 3)
    loss_ref, ref = mlp.loss_and_grads(params, X, t)
    assert abs(loss - loss_ref) <= 1e-6 * loss_ref
    for name, got, r in tensors(g, ref):
        d = np.abs(got - r)
        assert np.linalg.norm(d) <= 1e-6 * np.linalg.norm(r), (name, np.linalg.norm(d) / np.linalg.norm(r))
        worst = (d / np.maximum(np.abs(r), 1e-2 * np.abs(r).max())).max()
        assert worst <= 1e-4, (name, worst)


# the optimiser's constants as the device holds them (FP32 values)
HYP = dict(lr=float(np.float32(1e-3)), b1=float(np.float32(0.9)), b2=float(np.float32(0.999)),
           eps=float(np.float32(1e-8)), wd=float(np.float32(1e-4)))


def ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def step_error_bound(ref, p0, m1, m2, g, t):
    """FP32 error of one AdamW step, per element: the step's update carries
    one rounding in each of the bias corrections' divisions, the square
    root, the epsilon sum, the division and the learning-rate product, and
    the second moment's bias correction 1 - beta2^t inherits powf's error (at
    most 4 units in its last place, shrunk by the cancellation to 2.3
    relative units at t = 1000, halved by the root): 8 units in the last
    place of the update.  The new first moment b1 m + (1 - b1) g is formed
    with two roundings of its terms, an absolute error 2 u (b1 |m| +
    (1 - b1) |g|) that the step carries as lr / (c1 (sqrt(v / c2) + eps))
    times that (it dominates where the two terms nearly cancel).  One unit of
    the parameter for the final subtraction."""
    u = 2.0 ** -24
    b1, b2, lr, eps = HYP["b1"], HYP["b2"], HYP["lr"], HYP["eps"]
    c1, c2 = 1.0 - b1 ** t, 1.0 - b2 ** t
    v = b2 * m2 + (1.0 - b2) * g * g
    carried = lr * 2 * u * (b1 * np.abs(m1) + (1.0 - b1) * np.abs(g)) / c1 / (np.sqrt(v / c2) + eps)
    return 8.0 * ulp32(ref - p0) + ulp32(ref) + carried


@pytest.mark.parametrize("t_before", [0, 999])
def test_adamw_step_matches_oracle(P, t_before):
    """One step from the same FP32 parameters and moments, with t_before
    steps already taken (so the bias correction is that of step 1 or of
    step 1000)."""
    rng = np.random.default_rng(21 + t_before)
    params = [(f32(W), f32(b)) for W, b in mlp.init_params(48, 256, 4, seed=3)]
    p0 = mlp.flatten(params)
    n = p0.size
    m1 = f32(rng.standard_normal(n) * 1e-3) if t_before else np.zeros(n)
    m2 = f32(np.abs(rng.standard_normal(n)) * 1e-6) if t_before else np.zeros(n)
    g = f32(rng.standard_normal(n) * 1e-2)
    with P.Surrogate(256, 4) as S:
        S.set_params(p0, np.array([0.0, 1.0]))
        S.set_adam_state(m1, m2, t_before)
        S.adamw_step(g, lr=1e-3, weight_decay=1e-4)
        got = S.params()[0].astype(np.float64)
        m1g, m2g, tg = S.adam_state()
    assert tg == t_before + 1
    M1, M2 = mlp.unflatten(m1), mlp.unflatten(m2)
    state = [[(M1[l][0].copy(), M2[l][0].copy()), (M1[l][1].copy(), M2[l][1].copy())] for l in range(len(M1))]
    ref = mlp.flatten(mlp.adamw_step(mlp.unflatten(p0), mlp.unflatten(g), state, t_before + 1, **HYP))
    bound = step_error_bound(ref, p0, m1, m2, g, t_before + 1)
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, (ratio.max(), int(ratio.argmax()))
    m1r = mlp.flatten([(state[l][0][0], state[l][1][0]) for l in range(len(state))])
    m2r = mlp.flatten([(state[l][0][1], state[l][1][1]) for l in range(len(state))])
    u = 2.0 ** -24
    assert np.all(np.abs(m1g - m1r) <= 2 * u * (0.9 * np.abs(m1) + 0.1 * np.abs(g)))
    assert np.all(np.abs(m2g - m2r) <= 2 * u * m2r)


def test_adamw_1000_steps_drift(P):
    """1000 chained steps with fresh gradients: the FP32 parameters stay
    within the drift that FP32 moments allow.  The second moment's EMA
    carries a relative FP32 error up to u / (1 - beta2) = 6e-5, half of it
    through the square root into each step's update of size lr; summed over
    n steps, at most n lr u / (1 - beta2) / 2 = 3e-5 per element."""
    rng = np.random.default_rng(11)
    p0 = mlp.flatten([(f32(W), f32(b)) for W, b in mlp.init_params(48, 256, 4, seed=3)])
    pref = mlp.unflatten(p0.copy())
    state = mlp.zero_state(pref)
    with P.Surrogate(256, 4) as S:
        S.set_params(p0, np.array([0.0, 1.0]))
        for step in range(1, 1001):
            g = f32(rng.standard_normal(p0.size) * 1e-2)
            S.adamw_step(g, lr=1e-3, weight_decay=1e-4)
            pref = mlp.adamw_step(pref, mlp.unflatten(g), state, step, **HYP)
        got = S.params()[0].astype(np.float64)
    ref = mlp.flatten(pref)
    u, b2, lr, n = 2.0 ** -24, 0.999, 1e-3, 1000
    assert np.abs(got - ref).max() <= n * lr * u / (1 - b2) / 2
    assert np.linalg.norm(ref - p0) > 0.1 * np.linalg.norm(p0)  # the parameters did move
