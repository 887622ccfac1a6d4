"""Pins of the FP64 surrogate MLP oracle: finite differences, torch autograd
(float64) and torch's AdamW (float64).  CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def small(seed=0, in_dim=48, width=16, depth=3):
    return mlp.init_params(in_dim, width, depth, seed)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = small()
    X = rng.standard_normal((7, 48))
    t = rng.standard_normal(7)
    loss, grads = mlp.loss_and_grads(params, X, t)
    vec = mlp.flatten(params)
    g = mlp.flatten(grads)
    idx = rng.choice(vec.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        vp, vm = vec.copy(), vec.copy()
        vp[i] += h
        vm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unflatten(vp, 48, 16, 3), X, t)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(vm, 48, 16, 3), X, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def _torch_model(params):
    layers = []
    for l, (W, b) in enumerate(params):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
        if l < len(params) - 1:
            layers.append(torch.nn.GELU())
    return torch.nn.Sequential(*layers)


def test_forward_and_backward_match_torch_autograd():
    rng = np.random.default_rng(1)
    params = mlp.init_params(seed=3)
    X = rng.standard_normal((33, 48))
    t = rng.standard_normal(33)
    net = _torch_model(params)
    y_t = net(torch.from_numpy(X))[:, 0]
    loss_t = torch.mean((y_t - torch.from_numpy(t)) ** 2)
    loss_t.backward()
    y, _ = mlp.forward(params, X)
    loss, grads = mlp.loss_and_grads(params, X, t)
    np.testing.assert_allclose(y, y_t.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(loss - loss_t.item()) < 1e-12
    lin = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (gW, gb), m in zip(grads, lin):
        np.testing.assert_allclose(gW, m.weight.grad.numpy(), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(gb, m.bias.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_adamw_matches_torch():
    rng = np.random.default_rng(2)
    params = small(seed=5)
    X = rng.standard_normal((20, 48))
    t = rng.standard_normal(20)
    net = _torch_model(params)
    opt = torch.optim.AdamW(net.parameters(), lr=3e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.0)
    state = mlp.zero_state(params)
    for step in range(1, 6):
        opt.zero_grad()
        loss_t = torch.mean((net(torch.from_numpy(X))[:, 0] - torch.from_numpy(t)) ** 2)
        loss_t.backward()
        opt.step()
        _, grads = mlp.loss_and_grads(params, X, t)
        params = mlp.adamw_step(params, grads, state, step, lr=3e-3, wd=0.0)
    lin = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (W, b), m in zip(params, lin):
        np.testing.assert_allclose(W, m.weight.detach().numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(b, m.bias.detach().numpy(), rtol=1e-9, atol=1e-12)


def test_adamw_decoupled_decay_on_weights_only():
    # zero gradients: Adam's update vanishes, only lr * wd * W remains, biases untouched
    params = small(seed=6)
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    out = mlp.adamw_step(params, zeros, mlp.zero_state(params), 1, lr=0.1, wd=0.5)
    for (W, b), (W2, b2) in zip(params, out):
        np.testing.assert_allclose(W2, W * (1 - 0.05))
        np.testing.assert_allclose(b2, b)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-39, 65504.0])
    q = mlp.bf16(x)
    assert q[0] == 1.0
    assert q[1] == 1.0  # tie -> even mantissa
    assert q[2] == 1.0 + 2 ** -7  # above the midpoint rounds up
    assert q[3] == -2.5
    assert q[5] == 65536.0
    normal = np.abs(x) > 1.2e-38  # subnormals keep fewer significant bits
    assert np.all(np.abs(q - x)[normal] <= np.abs(x)[normal] * 2 ** -8)


def test_features_layout():
    th = np.array([[0.0, 1.0, 2.0]])
    x = mlp.features(th, [0, 0, 0], [2, 2, 2], np.arange(16))
    np.testing.assert_allclose(x[0, :3], [-1, 0, 1])
    assert np.all(x[0, 3:32] == 0)
    np.testing.assert_allclose(x[0, 32:], np.arange(16))


def test_targets_closed_forms_and_order():
    e = math.e
    # 1 + J + 10 class = 1, e, e^3
    t = mlp.targets([0.0, e - 1, e ** 3 - 11, np.inf, np.nan, -3.0, 5.0],
                    [0, 0, 1, 2, 0, 2, 3])
    np.testing.assert_allclose(t[:3], [0.0, 1.0, 3.0], rtol=0, atol=1e-14)
    assert t[3] == t[4] == pytest.approx(13.815511557963774, abs=1e-12)  # ln(1 000 001)
    assert t[5] == pytest.approx(math.log(21.0), abs=1e-15)  # a negative cost counts as 0
    assert t[6] == pytest.approx(math.log(36.0), abs=1e-15)
    # costs below 10: sorted by (class, J) gives increasing targets
    rng = np.random.default_rng(0)
    J = rng.uniform(0, 9.99, 500)
    c = rng.integers(0, 4, 500)
    order = np.lexsort((J, c))
    assert np.all(np.diff(mlp.targets(J, c)[order]) > 0)


def _bf16_torch(x):
    """Round a float64 tensor to BF16 and back (torch's own conversion,
    round to nearest even)."""
    return x.to(torch.bfloat16).to(torch.float64)


class _RoundFwd(torch.autograd.Function):
    """BF16 rounding of a stored operand: rounds the value, passes the
    gradient through unchanged."""

    @staticmethod
    def forward(ctx, x):
        return _bf16_torch(x)

    @staticmethod
    def backward(ctx, g):
        return g


class _RoundBwd(torch.autograd.Function):
    """BF16 rounding of a stored gradient: identity forward, rounds the
    gradient flowing back."""

    @staticmethod
    def forward(ctx, x):
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return _bf16_torch(g)


def test_bf16_emulating_backward_matches_autograd_through_rounding_ops():
    """The emulated backward against torch autograd on a network whose
    stored values pass through rounding ops: inputs, weights and hidden
    activations rounded going forward, hidden-layer gradients dz rounded
    going back, the output layer's gradient left in full precision.  Also
    different from the exact gradients by far more than rounding order, so
    a rounding point left out or added fails."""
    rng = np.random.default_rng(5)
    params = mlp.init_params(48, 32, 3, seed=4)
    X = rng.uniform(-1.5, 1.5, (40, 48))
    t = rng.standard_normal(40)
    a = _RoundFwd.apply(torch.from_numpy(X))
    Ws, bs = [], []
    for l, (W, b) in enumerate(params):
        Wt = torch.from_numpy(W.copy()).requires_grad_(True)
        bt = torch.from_numpy(b.copy()).requires_grad_(True)
        Ws.append(Wt)
        bs.append(bt)
        z = a @ _RoundFwd.apply(Wt).T + bt
        if l < len(params) - 1:
            z = _RoundBwd.apply(z)
            a = _RoundFwd.apply(0.5 * z * (1.0 + torch.special.erf(z / math.sqrt(2.0))))
        else:
            y = z[:, 0]
    loss_t = torch.mean((y - torch.from_numpy(t)) ** 2)
    loss_t.backward()
    loss, grads = mlp.loss_and_grads(params, X, t, emulate_bf16=True)
    assert abs(loss - loss_t.item()) < 1e-12
    _, exact = mlp.loss_and_grads(params, X, t)
    far = 0.0
    for (gW, gb), (eW, eb), Wt, bt in zip(grads, exact, Ws, bs):
        np.testing.assert_allclose(gW, Wt.grad.numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(gb, bt.grad.numpy(), rtol=1e-9, atol=1e-12)
        far = max(far, np.abs(gW - eW).max() / np.abs(eW).max())
    assert far > 1e-4
