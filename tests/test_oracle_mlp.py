"""Pins of the oracle's MLP: backward pass and input tangent against finite differences, one Adam step by hand."""
import numpy as np

from oracle import mlp


def _setup(seed=0, H=8, F=5, B=7):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(H, F, rng)
    params["b2"] = rng.standard_normal(H) * 0.3
    params["b3"] = rng.standard_normal(F) * 0.3
    t = rng.random(B)
    target = rng.standard_normal((B, F))
    return params, t, target


def test_backward_matches_finite_differences():
    params, t, target = _setup()
    loss, g = mlp.loss_and_grads(params, t, target)
    h = 1e-6
    for k, v in params.items():
        flat = v.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 9)):
            p1 = {kk: vv.copy() for kk, vv in params.items()}
            p2 = {kk: vv.copy() for kk, vv in params.items()}
            p1[k].reshape(-1)[idx] += h
            p2[k].reshape(-1)[idx] -= h
            fd = (mlp.loss_and_grads(p1, t, target)[0] - mlp.loss_and_grads(p2, t, target)[0]) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_input_tangent_matches_finite_differences():
    params, t, _ = _setup(1)
    _, dy, _ = mlp.forward(params, t, tangent=True)
    h = 1e-6
    fd = (mlp.forward(params, t + h)[0] - mlp.forward(params, t - h)[0]) / (2 * h)
    assert np.allclose(dy, fd, atol=1e-8)


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-9)


def test_first_adam_step_is_lr_times_sign():
    # with bias correction, the first step is lr * g / (|g| + eps)
    params, t, target = _setup(2)
    _, g = mlp.loss_and_grads(params, t, target)
    new = mlp.adam_step({k: v.copy() for k, v in params.items()}, g, {}, lr=1e-3)
    for k in params:
        assert np.allclose(params[k] - new[k], 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), atol=1e-15)


def _adam_run(grads, lr=1e-3, b1=0.9, b2=0.999):
    params = {"w": np.array([0.0])}
    state = {}
    steps = []
    for g in grads:
        before = params["w"].copy()
        params = mlp.adam_step(params, {"w": np.array([g])}, state, lr=lr, beta1=b1, beta2=b2, eps=0.0)
        steps.append(float((before - params["w"])[0]))
    return steps


def test_adam_constant_gradient_steps_are_lr():
    # a constant gradient g: m_t = g (1 - b1^t) and v_t = g^2 (1 - b2^t), so both bias-corrected moments equal g and
    # g^2 at every step and each step is exactly lr sign(g); a wrong power or beta in either correction breaks this
    # from the second step on
    for g in (0.37, -2.5):
        for s in _adam_run([g] * 4):
            assert abs(s - 1e-3 * np.sign(g)) <= 1e-15


def test_adam_alternating_and_growing_gradients_closed_forms():
    b1, b2, lr = 0.9, 0.999, 1e-3
    # g, -g, g: v_hat = g^2 throughout; m_hat is the normalised geometric sum of the alternating sequence
    g = 0.8
    s = _adam_run([g, -g, g], lr, b1, b2)
    assert abs(s[0] - lr) <= 1e-15
    assert abs(s[1] - (-lr * (1 - b1) / (1 + b1))) <= 1e-15
    assert abs(s[2] - lr * (b1 * b1 - b1 + 1) / (1 + b1 + b1 * b1)) <= 1e-15
    # g, 2g: m_hat = g (b1 + 2) / (1 + b1) and v_hat = g^2 (b2 + 4) / (1 + b2) at step 2
    s = _adam_run([g, 2 * g], lr, b1, b2)
    assert abs(s[1] - lr * (b1 + 2) / (1 + b1) * np.sqrt((1 + b2) / (b2 + 4))) <= 1e-15
    # g, 0, 0: the gradient's second moment decays with b2 and the momentum with b1
    s = _adam_run([g, 0.0, 0.0], lr, b1, b2)
    t = 3
    m_hat = (1 - b1) * b1 ** 2 * g / (1 - b1 ** t)
    v_hat = (1 - b2) * b2 ** 2 * g * g / (1 - b2 ** t)
    assert abs(s[2] - lr * m_hat / np.sqrt(v_hat)) <= 1e-15
