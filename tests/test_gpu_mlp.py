"""Learned radial surrogate and the exact per-pair radial path on the GPU.

* training kernels: loss and parameter gradients of one batch against the oracle's FP64 backward pass (1e-4);
* targets: the FP64 exact integrals (interpolated on a dense FP64 spline) against the oracle (1e-10);
* tensor-core inference (BF16 weights and activations, FP32 accumulation) against the oracle's FP64 forward;
* EXACT radial mode (1F1 + downward recurrence per pair, FP64) against the oracle: c within 1e-5, forces 1e-4;
* a trained network: its fit error against the exact integrals, and what it gains over the exact path.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import mlp as omlp  # noqa: E402
from oracle import radial as oradial  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import (System, config_tiny, linear_weights, mlp_initial_params, mlp_training_draws,  # noqa: E402
                   random_cell_atoms)
from tests.gpu_common import block_rel_err  # noqa: E402

H = 64


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _as_dict(p, F):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, 1)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (F, H)), ("b3", (F,))):
        size = int(np.prod(shape))
        out[name] = p[o:o + size].reshape(shape)
        o += size
    assert o == p.size
    return out


def _flat(d):
    return np.concatenate([d[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def _system(hyp, n_atoms=120, seed=41):
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (n_atoms / 0.06) ** (1 / 3)
    pos = random_cell_atoms(n_atoms, np.eye(3) * L, 1.6, rng)
    labels = hyp["species"]
    spe = np.asarray(labels, np.int32)[rng.integers(0, len(labels), n_atoms)]
    return System(pos, spe, (np.eye(3) * L)[None], np.ones((1, 3), np.int32), np.array([0, n_atoms], np.int32), dict(hyp))


SMALL = dict(r_cut=5.0, sigma=0.5, n_max=4, l_max=3, smooth_width=0.5, species=[1, 6])
MLPCFG = dict(r_cut=6.0, sigma=0.5, n_max=16, l_max=12, smooth_width=0.5, species=[1, 5, 6, 7, 8, 9, 15, 16])


def test_training_gradients_match_oracle(rg):
    import torch

    calc = rg.SoapCalculator(**SMALL)
    F = calc.n_max * (calc.l_max + 1)
    p0 = mlp_initial_params(H, F, seed=3)
    rng = np.random.default_rng(5)
    p0 = p0 + (rng.standard_normal(p0.size) * 0.05).astype(np.float32)  # non-zero biases everywhere
    calc.mlp_set_params(p0, np.ones(F, np.float32))
    t = rng.random(256).astype(np.float32)
    y = rng.standard_normal((256, F)).astype(np.float32)
    g, loss = calc.mlp_gradients(torch.tensor(t, device="cuda"), torch.tensor(y, device="cuda"))
    loss_ref, g_ref = omlp.loss_and_grads(_as_dict(p0, F), t.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    gd = _as_dict(g.cpu().numpy(), F)
    for k in g_ref:
        assert np.max(np.abs(gd[k] - g_ref[k])) <= 1e-4 * np.max(np.abs(g_ref[k])), k


def test_three_adam_steps_match_oracle(rg):
    # three steps on one batch, so the second-moment recurrence and both bias corrections enter (the first step
    # alone is lr sign(g) whatever they are)
    import torch

    calc = rg.SoapCalculator(**SMALL)
    F = calc.n_max * (calc.l_max + 1)
    p0 = mlp_initial_params(H, F, seed=4)
    calc.mlp_set_params(p0, np.ones(F, np.float32))
    rng = np.random.default_rng(6)
    t = rng.random(128).astype(np.float32)
    y = rng.standard_normal((128, F)).astype(np.float32)
    order = torch.arange(128, dtype=torch.int64, device="cuda")
    calc.mlp_train(torch.tensor(t, device="cuda"), torch.tensor(y, device="cuda"), order, batch=128, steps=3, lr_max=1e-3,
                   lr_min=1e-3)
    p1, _ = calc.mlp_get_params()
    ref = _as_dict(p0, F)
    state = {}
    for _ in range(3):
        g = omlp.loss_and_grads(ref, t.astype(np.float64), y.astype(np.float64))[1]
        ref = omlp.adam_step(ref, g, state, lr=1e-3)
    assert np.max(np.abs(p1 - _flat(ref))) <= 6e-6


def test_targets_are_the_exact_integrals(rg):
    import torch

    calc = rg.SoapCalculator(**MLPCFG)
    r = np.random.default_rng(7).uniform(0.0, 6.0, 300)
    tgt, scale = calc.mlp_targets(torch.tensor(r))
    ref = oradial.integrals(r, 6.0, 0.5, 16, 12)                      # [n, n_max, l+1]
    ref = np.transpose(ref, (0, 2, 1)).reshape(len(r), -1)          # f = l n_max + n
    got = tgt.cpu().numpy().astype(np.float64) * scale[None, :]
    # at n_max = 16 the two FP64 S^-1/2 (GPU Jacobi, oracle LAPACK) differ by ~5e-7 (cond S = 5.7e10); FP32
    # storage of the scaled target adds 6e-8 and the dense FP64 spline 1e-14
    assert np.max(np.abs(got - ref)) <= 3e-6 * np.max(np.abs(ref))


def test_tensor_core_inference_matches_fp64_forward(rg):
    calc = rg.SoapCalculator(**MLPCFG)
    F = calc.n_max * (calc.l_max + 1)
    p0 = mlp_initial_params(H, F, seed=8)
    rng = np.random.default_rng(9)
    scale = rng.uniform(0.5, 2.0, F).astype(np.float32)
    calc.mlp_set_params(p0, scale)
    r = rng.uniform(0.0, 6.0, 1000).astype(np.float32)
    out, dout = calc.mlp_eval(r, derivative=True)
    y, dy, _ = omlp.forward(_as_dict(p0, F), r.astype(np.float64) / 6.0, tangent=True)
    y_ref, dy_ref = y * scale, dy * scale / 6.0
    e_y = np.max(np.abs(out.cpu().numpy() - y_ref)) / np.max(np.abs(y_ref))
    e_dy = np.max(np.abs(dout.cpu().numpy() - dy_ref)) / np.max(np.abs(dy_ref))
    print(f"bf16 inference: value error {e_y:.2e}, derivative error {e_dy:.2e} (relative to the max)")
    # bfloat16 activations and weights: 8 significant bits per operand, summed over 64 inputs twice
    assert e_y <= 2e-2 and e_dy <= 3e-2


def test_exact_radial_mode_matches_oracle(rg):
    s = config_tiny()
    h = osoap.Hypers(**s.hypers)
    calc = rg.SoapCalculator(**s.hypers, radial="exact")
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c = calc.spherical_expansion(ds, pairs).cpu().numpy()
    assert block_rel_err(c, osoap.spherical_expansion(s, h), 2) <= 1e-5


def test_exact_radial_forces_match_oracle(rg):
    import torch

    from paper_2101_08814_gb300.autograd import LinearSoapEnergy

    s = _system(SMALL, n_atoms=60, seed=2)
    h = osoap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    calc = rg.SoapCalculator(**s.hypers, radial="exact")
    _, f, v = LinearSoapEnergy(calc, torch.tensor(w, dtype=torch.float32))(rg.DeviceSystem.from_numpy(s))
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    assert np.max(np.abs(f.cpu().numpy() - F_ref)) <= 1e-4 * np.max(np.abs(F_ref))
    assert np.max(np.abs(v.cpu().numpy() - V_ref)) <= 1e-4 * np.max(np.abs(V_ref))


def _train(rg, hyp, n_samples, steps, batch=2048, seed=22):
    import torch

    calc = rg.SoapCalculator(**hyp)
    F = calc.n_max * (calc.l_max + 1)
    r, order = mlp_training_draws(n_samples, hyp["r_cut"], batch, steps, seed=seed)
    tgt, scale = calc.mlp_targets(torch.tensor(r))
    calc.mlp_set_params(mlp_initial_params(H, F, seed=seed + 1), scale)
    t = torch.tensor(r / hyp["r_cut"], dtype=torch.float32, device="cuda")
    loss = calc.mlp_train(t, tgt, torch.tensor(order, device="cuda"), batch=batch, steps=steps, lr_max=3e-3, lr_min=1e-5,
                          total_steps=steps)
    return calc, scale, loss.cpu().numpy()


def test_trained_network_fits_and_gains_over_the_exact_path(rg, tmp_path):
    import torch

    calc, scale, loss = _train(rg, MLPCFG, n_samples=1 << 16, steps=3000)
    assert loss[-50:].mean() < 0.05 * loss[:10].mean()
    r = np.random.default_rng(10).uniform(0.0, 6.0, 2000)
    ref = np.transpose(oradial.integrals(r, 6.0, 0.5, 16, 12), (0, 2, 1)).reshape(len(r), -1)
    got = calc.mlp_eval(r.astype(np.float32)).cpu().numpy()
    fit = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"MLP fit after 3000 steps: max error {fit:.2e} of max |I|, final loss {loss[-1]:.2e}")
    assert fit < 0.1
    # checkpoint round trip
    path = tmp_path / "mlp.bin"
    calc.mlp_save(path)
    other = rg.SoapCalculator(**MLPCFG)
    other.mlp_load(path)
    assert np.array_equal(other.mlp_get_params()[0], calc.mlp_get_params()[0])
    # what the network gains: coefficients of the same system through the exact per-pair path and the MLP path
    s = _system(MLPCFG, n_atoms=400, seed=12)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    times = {}
    cs = {}
    for mode in ("exact", "mlp", "spline"):
        calc.set_radial(mode)
        calc.spherical_expansion(ds, pairs)
        calc.sync()
        t0 = time.perf_counter()
        for _ in range(3):
            c = calc.spherical_expansion(ds, pairs)
        calc.sync()
        times[mode] = (time.perf_counter() - t0) / 3
        cs[mode] = c.cpu().numpy()
    err_mlp = block_rel_err(cs["mlp"], cs["exact"], 2)
    err_spl = block_rel_err(cs["spline"], cs["exact"], 2)
    print(f"expansion of {s.n_atoms} centres: exact {times['exact'] * 1e3:.2f} ms, MLP {times['mlp'] * 1e3:.2f} ms, "
          f"spline {times['spline'] * 1e3:.2f} ms; coefficient error vs exact: MLP {err_mlp:.2e}, spline {err_spl:.2e}")
    assert times["mlp"] < times["exact"] / 3
    assert err_spl <= 1e-5
