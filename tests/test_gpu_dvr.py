"""GPU DVR radial basis (Eq. rad-int-dvr) against the FP64 oracle: the exact FP64 table, the spline built on it,
c and p on the tiny and two-species workloads, the per-pair exact mode and the forces.

Tolerances as for the GTO basis: 1e-12 relative for the FP64 table (1e-11 for its derivative), 1e-5 per block for
c and p on the FP32 path, 1e-4 for forces and virial.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import dvr as odvr  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import config_tiny, linear_weights, small_cell_system  # noqa: E402
from tests.gpu_common import block_rel_err, ps_blocks  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _run(rg, system, layout="packed", **over):
    h = dict(system.hypers, basis="dvr", **over)
    calc = rg.SoapCalculator(**h)
    ds = rg.DeviceSystem.from_numpy(system)
    pairs = calc.neighbours(ds)
    c = calc.spherical_expansion(ds, pairs)
    p = calc.power_spectrum(c, layout=layout)
    calc.sync()
    return calc, c.cpu().numpy(), p.cpu().numpy()


def test_dvr_table_fp64_matches_oracle(rg):
    import torch

    for hyp in (dict(r_cut=5.0, sigma=0.5, n_max=8, l_max=6), dict(r_cut=6.0, sigma=0.3, n_max=16, l_max=12),
                dict(r_cut=4.0, sigma=0.6, n_max=3, l_max=15)):
        calc = rg.SoapCalculator(**hyp, species=[1], basis="dvr")
        # r = 0 (series side), a point just above the series switch, and a grid across the cutoff
        r = np.concatenate([[0.0, 2e-5], np.linspace(1e-3, hyp["r_cut"], 95)])
        I, dI = calc.radial_exact_fp64(torch.tensor(r), derivative=True)
        Ir, dIr = odvr.integrals(r, hyp["r_cut"], hyp["sigma"], hyp["n_max"], hyp["l_max"], derivative=True)
        assert np.max(np.abs(I.cpu().numpy() - Ir)) <= 1e-12 * np.max(np.abs(Ir))
        assert np.max(np.abs(dI.cpu().numpy() - dIr)) <= 1e-11 * np.max(np.abs(dIr))
        # per n, relative to that function's own scale (the outer nodes are small inside r_cut)
        scale = np.max(np.abs(Ir), axis=(0, 2))
        assert np.all(np.max(np.abs(I.cpu().numpy() - Ir), axis=(0, 2)) <= 1e-11 * scale)


def test_dvr_spline_meets_its_accuracy_target(rg):
    calc = rg.SoapCalculator(**dict(config_tiny().hypers, basis="dvr"))
    assert calc.info["spline_error"] <= 1e-8
    assert calc.info["spline_error_fp32"] <= 2e-6


def test_dvr_tiny_all_centres(rg):
    s = config_tiny()
    h = osoap.Hypers(**dict(s.hypers, basis="dvr"))
    _, c, p = _run(rg, s)
    c_ref = osoap.spherical_expansion(s, h)
    p_ref = osoap.power_spectrum(c_ref, h, "packed")
    assert block_rel_err(c, c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p, h.l_max), p_ref, 2) <= TOL


def test_dvr_small_cell_two_species_full_layout(rg):
    s = small_cell_system(seed=23, n_atoms=9, L=5.0, hypers=dict(r_cut=5.0, sigma=0.45, n_max=6, l_max=5,
                                                                 smooth_width=0.7, species=[1, 8]))
    h = osoap.Hypers(**dict(s.hypers, basis="dvr"))
    _, c, p = _run(rg, s, layout="full")
    c_ref = osoap.spherical_expansion(s, h)
    assert block_rel_err(c, c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p, h.l_max), osoap.power_spectrum(c_ref, h, "full"), 2) <= TOL


def test_dvr_exact_radial_mode(rg):
    s = config_tiny()
    h = osoap.Hypers(**dict(s.hypers, basis="dvr"))
    _, c, _ = _run(rg, s, radial="exact")
    c_ref = osoap.spherical_expansion(s, h, centres=[0, 9, 31])
    assert block_rel_err(c[[0, 9, 31]], c_ref, 2) <= TOL


def test_dvr_forces_and_virial(rg):
    import torch

    from paper_2101_08814_gb300.autograd import LinearSoapEnergy

    s = small_cell_system(seed=29, n_atoms=24, L=7.0, hypers=dict(r_cut=4.5, sigma=0.4, n_max=6, l_max=5,
                                                                  smooth_width=0.5, species=[1, 6]))
    h = osoap.Hypers(**dict(s.hypers, basis="dvr"))
    w = linear_weights(h.n_species, h.n_features("packed"), seed=6)
    calc = rg.SoapCalculator(**dict(s.hypers, basis="dvr"))
    model = LinearSoapEnergy(calc, torch.tensor(w, dtype=torch.float32))
    e, f, v = model(rg.DeviceSystem.from_numpy(s))
    calc.sync()
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    E_ref = osoap.total_energy(s, h, w)
    f, v = f.cpu().numpy(), v.cpu().numpy()
    assert abs(float(e.cpu()[0]) - E_ref) <= 1e-5 * abs(E_ref)
    assert np.max(np.abs(f - F_ref)) <= 1e-4 * np.max(np.abs(F_ref))
    assert np.max(np.abs(v - V_ref)) <= 1e-4 * np.max(np.abs(V_ref))


def test_unknown_basis_is_an_argument_error(rg):
    import ctypes as C

    from paper_2101_08814_gb300 import _lib

    sp = (C.c_int * 1)(1)
    h = _lib.Hypers(5.0, 0.5, 0.5, 4, 3, 1, C.cast(sp, C.POINTER(C.c_int)), 0, 1, 0, 1, 0.0, 0, 7)
    ctx = C.c_void_p()
    assert _lib.lib().rascal_create(C.byref(h), None, C.byref(ctx)) != 0
