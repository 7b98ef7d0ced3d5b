"""GPU radial table, spherical expansion and FP32 power spectrum against the FP64 oracle.

Tolerance (FP32 path): per (centre, species) block of c and per (centre, l) block of p,
max |gpu - oracle| / max |oracle| <= 1e-5.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import radial as oradial  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import System, config_batch, config_tiny, random_cell_atoms, small_cell_system  # noqa: E402
from tests.gpu_common import block_rel_err, ps_blocks  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _run(rg, system, layout="packed", **over):
    h = dict(system.hypers, **over)
    calc = rg.SoapCalculator(**h)
    ds = rg.DeviceSystem.from_numpy(system)
    pairs = calc.neighbours(ds)
    c = calc.spherical_expansion(ds, pairs)
    p = calc.power_spectrum(c, layout=layout)
    calc.sync()
    return calc, c.cpu().numpy(), p.cpu().numpy()


def test_radial_exact_fp64_matches_oracle(rg):
    import torch

    for hyp in (dict(r_cut=5.0, sigma=0.5, n_max=8, l_max=6), dict(r_cut=6.0, sigma=0.5, n_max=16, l_max=12),
                dict(r_cut=5.5, sigma=0.4, n_max=8, l_max=6)):
        calc = rg.SoapCalculator(**hyp, species=[1])
        r = np.linspace(0.0, hyp["r_cut"], 97)
        I, dI = calc.radial_exact_fp64(torch.tensor(r), derivative=True)
        Ir, dIr = oradial.integrals(r, hyp["r_cut"], hyp["sigma"], hyp["n_max"], hyp["l_max"], derivative=True)
        # the o-GTO transform amplifies FP64 rounding by up to cond(S)^1/2 (about 2e5 at n_max = 16); the
        # derivative is a difference of two G terms (Appendix A) and loses about two more digits to cancellation
        # at n_max = 16, cond(S) = 5.7e10 and either FP64 eigensolver is off by ~5e-7 in S^-1/2 (pinned in
        # test_oracle_radial against 40 digits), which carries into I^o
        tol = 1e-12 if hyp["n_max"] <= 8 else 2e-6
        assert np.max(np.abs(I.cpu().numpy() - Ir)) <= tol * np.max(np.abs(Ir))
        assert np.max(np.abs(dI.cpu().numpy() - dIr)) <= 100 * tol * np.max(np.abs(dIr))


def test_spline_meets_its_accuracy_target(rg):
    calc = rg.SoapCalculator(**config_tiny().hypers)
    assert calc.info["spline_error"] <= 1e-8
    assert calc.info["spline_error_fp32"] <= 2e-6
    assert calc.info["spline_intervals"] >= 64


def test_tiny_all_centres(rg):
    s = config_tiny()
    h = osoap.Hypers(**s.hypers)
    _, c, p = _run(rg, s)
    c_ref = osoap.spherical_expansion(s, h)
    p_ref = osoap.power_spectrum(c_ref, h, "packed")
    assert block_rel_err(c, c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p, h.l_max), p_ref, 2) <= TOL


def test_full_layout_and_raw_basis(rg):
    s = config_tiny()
    h = osoap.Hypers(**dict(s.hypers, orthonormal=False))
    _, c, p = _run(rg, s, layout="full", orthonormal=False)
    centres = [0, 5, 40]
    c_ref = osoap.spherical_expansion(s, h, centres=centres)
    p_ref = osoap.power_spectrum(c_ref, h, "full")
    assert block_rel_err(c[centres], c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p[centres], h.l_max), p_ref, 2) <= TOL


def test_small_cell_self_images_two_species(rg):
    s = small_cell_system(seed=21, n_atoms=9, L=5.0, hypers=dict(r_cut=5.0, sigma=0.45, n_max=6, l_max=5, smooth_width=0.7,
                                                                 species=[1, 8]))
    h = osoap.Hypers(**s.hypers)
    _, c, p = _run(rg, s)
    c_ref = osoap.spherical_expansion(s, h)
    assert block_rel_err(c, c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p, h.l_max), osoap.power_spectrum(c_ref, h, "packed"), 2) <= TOL


def test_include_center(rg):
    s = config_tiny()
    h = osoap.Hypers(**dict(s.hypers, include_center=True))
    _, c, _ = _run(rg, s, include_center=True)
    c_ref = osoap.spherical_expansion(s, h, centres=[3, 7])
    assert block_rel_err(c[[3, 7]], c_ref, 2) <= TOL


def test_many_species_several_rounds(rg):
    # 8 species with n_max = 16, l_max = 12: the kernel accumulates the species in several rounds
    rng = np.random.Generator(np.random.PCG64(77))
    L = 15.0
    pos = random_cell_atoms(200, np.eye(3) * L, 1.6, rng)
    labels = [1, 5, 6, 7, 8, 9, 15, 16]
    s = System(pos, np.asarray(labels, np.int32)[rng.integers(0, 8, 200)], (np.eye(3) * L)[None], np.ones((1, 3), np.int32),
               np.array([0, 200], np.int32), dict(r_cut=6.0, sigma=0.5, n_max=16, l_max=12, smooth_width=0.5, species=labels))
    h = osoap.Hypers(**s.hypers)
    _, c, p = _run(rg, s)
    centres = [0, 99, 199]
    c_ref = osoap.spherical_expansion(s, h, centres=centres)
    assert block_rel_err(c[centres], c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p[centres], h.l_max), osoap.power_spectrum(c_ref, h, "packed"), 2) <= TOL


def test_batch_full_size_sampled(rg):
    s = config_batch()
    h = osoap.Hypers(**s.hypers)
    calc, c, p = _run(rg, s)
    rng = np.random.default_rng(1)
    centres = np.concatenate([[0, s.n_atoms - 1], rng.choice(s.n_atoms, 14, replace=False)])
    c_ref = osoap.spherical_expansion(s, h, centres=centres)
    assert block_rel_err(c[centres], c_ref, 2) <= TOL
    assert block_rel_err(ps_blocks(p[centres], h.l_max), osoap.power_spectrum(c_ref, h, "packed"), 2) <= TOL
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(p))


def test_fused_soap_equals_separate_calls(rg):
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c1 = calc.spherical_expansion(ds, pairs)
    p1 = calc.power_spectrum(c1)
    c2, p2 = calc.soap(ds, pairs)
    assert np.array_equal(c1.cpu().numpy(), c2.cpu().numpy())
    assert np.max(np.abs(p1.cpu().numpy() - p2.cpu().numpy())) <= 1e-6 * np.max(np.abs(p1.cpu().numpy()))


@pytest.mark.parametrize("hyp_name", ["HYPERS_BATCH", "HYPERS_LARGE", "HYPERS_DIFF", "HYPERS_MLP"])
def test_shaped_instances_match_oracle(rg, hyp_name):
    # the hyper shapes with their own compiled instance of the fused FP32 kernel (compile-time n_max, l_max and
    # species count): fused c and p, PACKED and FULL, against the oracle, with a crowded centre (more pairs than one
    # staged chunk) and an isolated atom; the same system through the separate calls as a second check
    import synth

    hyp = dict(getattr(synth.structures, hyp_name))
    rng = np.random.Generator(np.random.PCG64(31))
    L = 30.0
    pos = np.concatenate([random_cell_atoms(70, np.eye(3) * 9.0, 1.05, rng) + 2.0, [[25.0, 25.0, 25.0]]])
    labels = hyp["species"]
    spe = np.asarray(labels, np.int32)[rng.integers(0, len(labels), len(pos))]
    s = System(pos, spe, (np.eye(3) * L)[None], np.zeros((1, 3), np.int32), np.array([0, len(pos)], np.int32), hyp)
    h = osoap.Hypers(**hyp)
    c_ref = osoap.spherical_expansion(s, h)
    calc = rg.SoapCalculator(**hyp)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    assert np.diff(pairs.offsets.cpu().numpy()).max() > 32
    # at n_max = 16 (cond(S) = 5.7e10) the FP64 S^-1/2 of the GPU and of the oracle agree only to ~5e-7 relative
    # (the oracle's own is pinned to 40 digits at that level); after the cancellation inside a crowded centre's
    # (species) block this reaches 2.2e-5 of the block's max, identically with the exact per-pair radial path and
    # with the runtime-shaped kernel, so the bar follows the basis transform there: 5e-5 for c, twice that for p
    tol_c = TOL if h.n_max <= 12 else 5e-5
    tol_p = TOL if h.n_max <= 12 else 1e-4
    for layout in ("packed", "full"):
        c, p = calc.soap(ds, pairs, layout=layout)
        p_sep = calc.power_spectrum(calc.spherical_expansion(ds, pairs), layout=layout)
        calc.sync()
        c, p, p_sep = c.cpu().numpy(), p.cpu().numpy(), p_sep.cpu().numpy()
        p_ref = osoap.power_spectrum(c_ref, h, layout).reshape(len(pos), h.l_max + 1, -1)
        assert block_rel_err(c, c_ref, 2) <= tol_c
        assert block_rel_err(ps_blocks(p, h.l_max), p_ref, 2) <= tol_p, layout
        assert block_rel_err(ps_blocks(p_sep, h.l_max), p_ref, 2) <= tol_p, layout
        assert np.all(c[-1] == 0.0) and np.all(p[-1] == 0.0)
    # the tensor-core forms and the coefficients-only call have their own instances for these shapes
    c_only = calc.spherical_expansion(ds, pairs).cpu().numpy()
    assert block_rel_err(c_only, c_ref, 2) <= tol_c
    p_ref = osoap.power_spectrum(c_ref, h, "packed").reshape(len(pos), h.l_max + 1, -1)
    for prec, tol in (("tf32x3", TOL), ("bf16", 2.0 ** -7)):
        try:
            c_tc, p_tc = calc.soap(ds, pairs, precision=prec)
            calc.sync()
        except rg.RascalError as e:  # TF32 hi/lo tiles of Q > 96 exceed shared memory: refused, not run
            assert e.code == rg._lib.RASCAL_E_UNSUPPORTED and prec == "tf32x3" and h.q > 96
            continue
        assert block_rel_err(c_tc.cpu().numpy(), c_ref, 2) <= tol_c, prec
        assert block_rel_err(ps_blocks(p_tc.cpu().numpy(), h.l_max), p_ref, 2) <= max(tol, tol_p), prec
    # selected packed features (the selection form's instance for the same shape)
    F = h.n_features("packed")
    sel = np.random.default_rng(3).choice(F, size=F // 7, replace=False).astype(np.int32)
    c_sel, p_sel = calc.soap_selected(ds, pairs, sel)
    calc.sync()
    assert np.array_equal(c_sel.cpu().numpy(), c_only)
    ref_sel = osoap.power_spectrum(c_ref, h, "packed").reshape(len(pos), -1)[:, sel]
    assert block_rel_err(p_sel.cpu().numpy(), ref_sel, 1) <= tol_p
    # forces and virial of the linear energy model through the gradient kernel's instance for the same shape
    import torch

    from paper_2101_08814_gb300.autograd import LinearSoapEnergy
    from synth import linear_weights

    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    _, f, v = LinearSoapEnergy(calc, torch.tensor(w, dtype=torch.float32))(ds)
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    assert np.max(np.abs(f.cpu().numpy() - F_ref)) <= 1e-4 * np.max(np.abs(F_ref))
    assert np.max(np.abs(v.cpu().numpy() - V_ref)) <= 1e-4 * np.max(np.abs(V_ref))
