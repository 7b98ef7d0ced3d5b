"""Parity on the large liquid-like workload (32 768 atoms, 3 species 2:1:1, 0.1 atoms/A^3, r_cut 6 A, about 90
neighbours per centre, n_max 10, l_max 8) at full size, on a seeded sample of centres the oracle computes one by one:
* neighbour lists of the sampled centres bit-exact;
* c within 1e-5 per (centre, species) block;
* p within 1e-5 per (centre, l) block for FP32 and TF32x3, BF16 within 2^-7 (block max) and 5e-3 (block Frobenius);
* forces and virial of the energy of the sampled centres only (dE/dp = the linear model's weights on those centres,
  zero elsewhere) within 1e-4 of their maximum.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import soap as osoap  # noqa: E402
from oracle.neighbours import neighbour_list  # noqa: E402
from synth import config_large, linear_weights  # noqa: E402
from tests.gpu_common import block_rel_err, ps_blocks  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def test_large_workload_sampled(rg):
    import torch

    s = config_large()
    h = osoap.Hypers(**s.hypers)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    rng = np.random.default_rng(8)
    centres = np.sort(np.concatenate([[0, s.n_atoms - 1], rng.choice(np.arange(1, s.n_atoms - 1), 14, replace=False)]))
    nl = neighbour_list(s, h.r_cut, centres)
    off = pairs.offsets.cpu().numpy()
    idx = np.concatenate([np.arange(off[c], off[c + 1]) for c in centres])
    assert np.array_equal(np.diff(off)[centres], np.diff(nl["offsets"]))
    assert np.array_equal(pairs.nbr_j.cpu().numpy()[idx], nl["nbr_j"])
    assert np.array_equal(pairs.shifts.cpu().numpy()[idx], nl["shifts"])
    assert np.diff(nl["offsets"]).mean() > 60
    c_ref = osoap.spherical_expansion(s, h, nl=nl)
    p_ref = osoap.power_spectrum(c_ref, h, "packed").reshape(len(centres), h.l_max + 1, -1)
    c32 = None
    for prec in ("fp32", "tf32x3", "bf16"):
        c, p = calc.soap(ds, pairs, precision=prec)
        calc.sync()
        cg = c.cpu().numpy()[centres]
        assert block_rel_err(cg, c_ref, 2) <= 1e-5, prec
        got = ps_blocks(p.cpu().numpy()[centres], h.l_max).astype(np.float64)
        err = block_rel_err(got, p_ref, 2)
        if prec == "bf16":
            assert err <= 2.0 ** -7, err
            fro = np.sqrt(np.sum((got - p_ref) ** 2, axis=-1) / np.maximum(np.sum(p_ref ** 2, axis=-1), 1e-300))
            assert np.max(fro) <= 5e-3, np.max(fro)
        else:
            assert err <= 1e-5, (prec, err)
        if prec == "fp32":
            c32 = c
    # forces and virial of the sampled centres' energy
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    a = h.species_index(s.species)
    gp = torch.zeros((s.n_atoms, h.n_features("packed")), dtype=torch.float32, device="cuda")
    gp[torch.as_tensor(centres, device="cuda")] = torch.tensor(w[a[centres]], dtype=torch.float32, device="cuda")
    F, V = calc.gradients(ds, pairs, c32, grad_ps=gp)
    F_ref, V_ref = osoap.energy_gradients(s, h, w, centres=centres, nl=nl)
    F, V = F.cpu().numpy(), V.cpu().numpy()
    assert np.max(np.abs(F - F_ref)) <= 1e-4 * np.max(np.abs(F_ref))
    assert np.max(np.abs(V - V_ref)) <= 1e-4 * np.max(np.abs(V_ref))
