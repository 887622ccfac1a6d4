"""FP64 reference of the cost-surrogate MLP -- TEST INFRASTRUCTURE.

The surrogate is not part of the paper (the task asks for it): an MLP
x -> y with x = [theta padded to 32 | 16 scene features], hidden layers
Linear + GELU (exact, erf form), a scalar linear output, trained by minibatch
AdamW on the mean squared error.  This module restates it in float64 numpy
with explicit chain-rule backward, plus an emulation of the library's BF16
rounding points (weights, layer inputs and activations rounded to BF16 with
round-to-nearest-even; products accumulated exactly here, in FP32 on the GPU).

Pins (tests/test_oracle_mlp.py): central finite differences of the FP64
loss, torch.autograd in float64, and torch.optim.AdamW in float64; the
BF16-emulating backward against torch.autograd run on the same rounded
operands (a hand-written chain through BF16-rounded tensors); the
regression targets at closed-form points (e - 1, e^3 - 11, a non-finite
cost, a negative cost) and their class-first order for costs below 10.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(in_dim=48, width=256, depth=4, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (the usual
    Linear-layer default), layers in order; W[l] has shape (out, in)."""
    rng = np.random.default_rng(seed)
    dims = [in_dim] + [width] * depth + [1]
    params = []
    for l in range(len(dims) - 1):
        bound = 1.0 / math.sqrt(dims[l])
        W = rng.uniform(-bound, bound, (dims[l + 1], dims[l]))
        b = rng.uniform(-bound, bound, dims[l + 1])
        params.append((W, b))
    return params


def forward(params, X, emulate_bf16=False):
    """y[M] and the cache (layer inputs and pre-activations)."""
    a = bf16(X) if emulate_bf16 else np.asarray(X, np.float64)
    acts, pre = [a], []
    for l, (W, b) in enumerate(params):
        Wq = bf16(W) if emulate_bf16 else W
        z = a @ Wq.T + b
        if l < len(params) - 1:
            pre.append(z)
            a = gelu(z)
            if emulate_bf16:
                a = bf16(a)
            acts.append(a)
        else:
            return z[:, 0], (acts, pre)


def loss_and_grads(params, X, t, emulate_bf16=False):
    """MSE loss mean((y - t)^2) and its gradient with respect to every W, b,
    by the chain rule: dL/dy = 2 (y - t) / M; for layer l with input a_l and
    pre-activation z_l, dL/dW_l = dz_l^T a_l, dL/db_l = sum over rows of dz_l
    and dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1}).

    emulate_bf16 rounds where the library's BF16 training path stores BF16
    values, with everything in between exact: the inputs, every weight
    matrix, every hidden activation (forward), and every hidden-layer
    gradient dz (backward; the output layer's dL/dy stays FP32).  Only the
    library's FP32 accumulation then differs."""
    q = bf16 if emulate_bf16 else (lambda v: v)
    y, (acts, pre) = forward(params, X, emulate_bf16=emulate_bf16)
    M = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dz = (2.0 / M) * r[:, None]  # dL/dz of the output layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (dz.T @ acts[l], dz.sum(0))
        if l > 0:
            dz = q((dz @ q(W)) * gelu_grad(pre[l - 1]))
    return loss, grads


def adamw_step(params, grads, state, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One decoupled-weight-decay Adam step (Loshchilov & Hutter): weight decay
    on W only; `state` holds the first and second moments; step counts from 1."""
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m, v = state[l][j]
            m = b1 * m + (1 - b1) * g
            v = b2 * v + (1 - b2) * g * g
            state[l][j] = (m, v)
            mh = m / (1 - b1 ** step)
            vh = v / (1 - b2 ** step)
            decay = wd if j == 0 else 0.0
            p = p - lr * decay * p - lr * mh / (np.sqrt(vh) + eps)
            new.append(p)
        out.append(tuple(new))
    return out


def zero_state(params):
    return [[(np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b))] for W, b in params]


def flatten(params):
    """Weights then bias of each layer, concatenated (the library's order)."""
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params])


def unflatten(vec, in_dim=48, width=256, depth=4):
    dims = [in_dim] + [width] * depth + [1]
    out, o = [], 0
    for l in range(len(dims) - 1):
        n, k = dims[l + 1], dims[l]
        W = vec[o:o + n * k].reshape(n, k)
        o += n * k
        b = vec[o:o + n]
        o += n
        out.append((W.copy(), b.copy()))
    return out


def features(theta, lo, hi, scene16):
    """x = [(clip(theta) - mid) / half-range padded with zeros to 32 | scene16];
    theta is clipped to its bounds as the rollout does."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    theta = np.clip(np.asarray(theta, np.float64), lo, hi)
    M, D = theta.shape
    x = np.zeros((M, 48))
    x[:, :D] = (theta - 0.5 * (lo + hi)) / (0.5 * (hi - lo))
    x[:, 32:48] = np.asarray(scene16, np.float64)[None, :]
    return x


def targets(J, cls):
    """Regression target of a simulated sample: log(1 + max(J, 0) + 10 class),
    and log(1 + 1e6) where the cost is not finite.  The class term ranks
    classes first as the CE key does while costs stay below 10; the
    logarithm compresses large costs."""
    J = np.asarray(J, np.float64)
    c = np.asarray(cls, np.float64)
    with np.errstate(invalid="ignore"):
        t = np.log1p(np.maximum(J, 0.0) + 10.0 * c)
    return np.where(np.isfinite(J), t, math.log1p(1e6))
