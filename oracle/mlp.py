"""A 1 -> H -> H -> F multilayer perceptron with SiLU activations, in FP64: forward, input tangent, the backward
pass of a mean-squared-error loss and one Adam step.

This is the learned stand-in for the radial integrals r -> {I^o_nl(r)}. The paper does not contain it; its
nearest hook is the remark that the radial basis is a target for numerical optimisation (end of Sec. 'Spline
optimization'). The oracle version exists to check the GPU training kernels' gradients.

Conventions: input t = r / r_scale; z1 = W1 t + b1, h1 = silu(z1), z2 = W2 h1 + b2, h2 = silu(z2),
y = W3 h2 + b3; silu(z) = z sigmoid(z). Loss L = mean over batch and outputs of (y - target)^2.
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def init_params(hidden: int, n_out: int, rng: np.random.Generator):
    return dict(
        W1=rng.standard_normal((hidden, 1)) * 1.0,
        b1=rng.uniform(-1.0, 1.0, hidden),
        W2=rng.standard_normal((hidden, hidden)) / np.sqrt(hidden),
        b2=np.zeros(hidden),
        W3=rng.standard_normal((n_out, hidden)) / np.sqrt(hidden),
        b3=np.zeros(n_out),
    )


def forward(params, t, tangent=False):
    t = np.asarray(t, dtype=np.float64).reshape(-1, 1)
    z1 = t @ params["W1"].T + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    cache = dict(t=t, z1=z1, h1=h1, z2=z2, h2=h2, y=y)
    if not tangent:
        return y, cache
    dz1 = np.broadcast_to(params["W1"][:, 0], z1.shape)
    dh1 = silu_grad(z1) * dz1
    dz2 = dh1 @ params["W2"].T
    dh2 = silu_grad(z2) * dz2
    dy = dh2 @ params["W3"].T
    return y, dy, cache


def loss_and_grads(params, t, target):
    y, cache = forward(params, t)
    B, F = y.shape
    diff = y - target
    loss = float(np.mean(diff * diff))
    dy = 2.0 * diff / (B * F)
    g = {}
    g["W3"] = dy.T @ cache["h2"]
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ params["W3"]
    dz2 = dh2 * silu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * silu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["t"]
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction; state holds m, v per parameter and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
