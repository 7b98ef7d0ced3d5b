"""Adversarial geometries on the GPU against the oracle:
* neighbours exactly on the +z and -z axes (the pole of the Y_lm recurrences and of their gradients): c within 1e-5
  per block, forces and virial within 1e-4;
* a single neighbour: p takes the closed form f^2 I_n1l I_n2l sqrt(2l+1)/(4 pi) in the neighbour's species block and
  is zero elsewhere, in every precision (FP32 and TF32x3 within 1e-5, BF16 within 2^-7 of the block maximum).
"""
from math import pi, sqrt

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import radial as oradial  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import System, linear_weights  # noqa: E402
from tests.gpu_common import block_rel_err  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


HYP = dict(r_cut=5.0, sigma=0.5, n_max=6, l_max=6, smooth_width=0.5, species=[1, 8])


def _cluster(pos, species):
    pos = np.asarray(pos, np.float64)
    return System(pos, np.asarray(species, np.int32), (np.eye(3) * 40.0)[None], np.zeros((1, 3), np.int32),
                  np.array([0, len(pos)], np.int32), dict(HYP))


def test_neighbours_on_the_z_axis(rg):
    import torch

    from paper_2101_08814_gb300.autograd import LinearSoapEnergy

    c0 = np.array([10.0, 10.0, 10.0])
    pos = [c0, c0 + [0, 0, 2.2], c0 + [0, 0, -3.1], c0 + [1.3, 0.4, 0.9], c0 + [0, 0, 4.7], c0 + [-1.7, 1.1, -1.2]]
    s = _cluster(pos, [1, 8, 1, 8, 8, 1])
    h = osoap.Hypers(**s.hypers)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c = calc.spherical_expansion(ds, pairs).cpu().numpy()
    assert block_rel_err(c, osoap.spherical_expansion(s, h), 2) <= 1e-5
    for prec in ("tf32x3", "bf16"):
        c2, _ = calc.soap(ds, pairs, precision=prec)
        calc.sync()
        assert block_rel_err(c2.cpu().numpy(), osoap.spherical_expansion(s, h), 2) <= 1e-5, prec
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    _, f, v = LinearSoapEnergy(calc, torch.tensor(w, dtype=torch.float32))(ds)
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    assert np.all(np.isfinite(f.cpu().numpy()))
    assert np.max(np.abs(f.cpu().numpy() - F_ref)) <= 1e-4 * np.max(np.abs(F_ref))
    assert np.max(np.abs(v.cpu().numpy() - V_ref)) <= 1e-4 * np.max(np.abs(V_ref))


def test_single_neighbour_closed_form(rg):
    d = np.array([0.9, -2.3, 1.6])
    s = _cluster([[10.0, 10.0, 10.0], [10.9, 7.7, 11.6]], [1, 8])
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    r = np.linalg.norm(d)
    f = osoap.cutoff(r, 5.0, 0.5)
    I = oradial.integrals(np.array([r]), 5.0, 0.5, 6, 6)[0]          # [n, l]
    n, Q = 6, 12
    for centre, block in ((0, 1), (1, 0)):  # the neighbour's species block: label 8 -> 1, label 1 -> 0
        ref = np.zeros((7, Q, Q))
        for l in range(7):
            ref[l, block * n:(block + 1) * n, block * n:(block + 1) * n] = \
                f * f * np.outer(I[:, l], I[:, l]) * sqrt(2 * l + 1) / (4 * pi)
        for prec in ("fp32", "tf32x3", "bf16"):
            _, p = calc.soap(ds, pairs, layout="full", precision=prec)
            calc.sync()
            got = p.cpu().numpy()[centre].reshape(7, Q, Q).astype(np.float64)
            err = block_rel_err(got, ref, 1)
            assert err <= (2.0 ** -7 if prec == "bf16" else 1e-5), (centre, prec, err)
            outside = np.ones((Q, Q), bool)
            outside[block * n:(block + 1) * n, block * n:(block + 1) * n] = False
            assert np.all(got[:, outside] == 0.0), (centre, prec)
