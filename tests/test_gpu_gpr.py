"""GPU sparse GPR model (Eq. sparse-gp, polynomial kernel, TF32 tensor cores) against the FP64 oracle.

Bounds. The sparse points are stored as the nearest TF32 values of M^ and the tensor core reads the FP32 features
with the low 13 mantissa bits dropped, so each product in k = p^ . M^ carries a relative error below 2^-10 + 2^-11;
for unit vectors |dk| <= (2^-10 + 2^-11) sum_q |p^_q M^_q| <= 2^-9.4, and |dE_i| <= zeta |dk| sum_I |x_I|
(|k| <= 1). Against an emulation of exactly that input rounding (FP64 arithmetic on the rounded inputs) only FP32
accumulation remains: F terms of size <= 1 summed in FP32, bounded here by 1e-5 sum_I |x_I| zeta.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import gpr as ogpr  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import System, config_tiny, gpr_sparse_draws, random_cell_atoms  # noqa: E402

U_IN = 2.0 ** -10 + 2.0 ** -11


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def tf32_nearest(a):
    """Nearest TF32 value (ties to even) of float32 values, as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0xFFF + ((u >> 13) & 1)) & ~np.uint64(0x1FFF)
    return u.astype(np.uint32).view(np.float32)


def tf32_trunc(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def _unit_tf32(M):
    """Unit-normalised sparse points rounded to TF32: the model stores exactly these values."""
    Mh = M / np.linalg.norm(M, axis=1, keepdims=True)
    return tf32_nearest(Mh).astype(np.float64)


def _emulated_energies(p32, cs, Mt, ms, x, zeta, rounding):
    """FP64 energies from the inputs as the tensor core sees them: features rounded by `rounding`, the norm from
    the FP32 features, sparse points already TF32, weights FP32."""
    pr = rounding(p32).astype(np.float64)
    nrm = np.sqrt(np.sum(p32.astype(np.float64) ** 2, axis=1))
    nrm = np.where(nrm > 0, nrm, 1.0)
    x32 = x.astype(np.float32).astype(np.float64)
    E = np.zeros(p32.shape[0])
    for s in np.unique(cs):
        rows, cols = np.flatnonzero(cs == s), np.flatnonzero(ms == s)
        if cols.size:
            E[rows] = ((pr[rows] @ Mt[cols].T / nrm[rows, None]) ** zeta) @ x32[cols]
    return E


def _grad_checks(g, p32, cs, Mt, ms, x, zeta, pm_exact):
    """dE/dp from the GPU against (i) FP64 arithmetic on the inputs as the tensor core sees them (truncated features
    for k, the FP32 factor W = x zeta k^(zeta-1) truncated to TF32, the stored sparse points), within FP32
    accumulation; (ii) the exact FP64 oracle, within the first-order propagation of the input rounding through
    dE/dp = (1/|p|) sum_I x_I zeta [k^(zeta-1) M^_I - k^zeta p^]:
        |dg_q| <= (1/|p|) sum_I |x_I| zeta [((zeta-1)|k|^(zeta-2) eps_k + u_W |k|^(zeta-1)) |M^_Iq|
                                             + zeta |k|^(zeta-1) eps_k |p^_q|],
    eps_k = 2^-9.4 (the bound on k), u_W = 2^-10 + 2^-11 (W truncated, M^ rounded), doubled for the neglected
    second-order terms. Returns the two worst ratios error / allowed."""
    p64 = p32.astype(np.float64)
    nrm = np.sqrt(np.sum(p64 ** 2, axis=1))
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 1.0)
    pr = tf32_trunc(p32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    worst_emul, worst_exact = 0.0, 0.0
    eps_k, u_w = 2.0 ** -9.4, 2.0 ** -10 + 2.0 ** -11
    for sp in np.unique(cs):
        rows, cols = np.flatnonzero(cs == sp), np.flatnonzero(ms == sp)
        if cols.size == 0:
            continue
        k = (pr[rows] @ Mt[cols].T) * inv[rows, None]
        W = tf32_trunc((x32[cols][None, :] * zeta * k ** (zeta - 1)).astype(np.float32)).astype(np.float64)
        E = (k ** zeta) @ x32[cols]
        ge = inv[rows, None] * (W @ Mt[cols]) - (zeta * E * inv[rows] ** 2)[:, None] * p64[rows]
        scale = inv[rows, None] * (np.abs(W) @ np.abs(Mt[cols])) + np.abs(zeta * E * inv[rows] ** 2)[:, None] * np.abs(p64[rows])
        # a W within FP32 accumulation error (relative 1e-5) of a TF32 step may be truncated to either neighbour
        Wf = (x32[cols][None, :] * zeta * k ** (zeta - 1)).astype(np.float32)
        amb = tf32_trunc((Wf * np.float32(1 - 1e-5)).astype(np.float32)) != tf32_trunc((Wf * np.float32(1 + 1e-5)).astype(np.float32))
        flip = inv[rows, None] * ((amb * 2.0 ** -9 * np.abs(Wf)) @ np.abs(Mt[cols]))
        worst_emul = max(worst_emul, float(np.max(np.abs(g[rows] - ge) / (1e-4 * scale + flip + 1e-30))))
        Mx = pm_exact[cols] / np.linalg.norm(pm_exact[cols], axis=1, keepdims=True)
        kx = (p64[rows] * inv[rows, None]) @ Mx.T
        gx = inv[rows, None] * ((x[cols][None, :] * zeta * kx ** (zeta - 1)) @ Mx) - \
            (zeta * ((kx ** zeta) @ x[cols]) * inv[rows])[:, None] * (p64[rows] * inv[rows, None])
        ak = np.abs(kx)
        a1 = (np.abs(x[cols]) * zeta)[None, :] * (((zeta - 1) * ak ** max(zeta - 2, 0) * eps_k if zeta > 1 else 0.0)
                                                   + u_w * ak ** (zeta - 1))
        a2 = (np.abs(x[cols]) * zeta * zeta)[None, :] * ak ** (zeta - 1) * eps_k
        bound = 2.0 * inv[rows, None] * (a1 @ np.abs(Mx) + (a2.sum(axis=1))[:, None] * np.abs(p64[rows] * inv[rows, None]))
        worst_exact = max(worst_exact, float(np.max(np.abs(g[rows] - gx) / (bound + 1e-30))))
    return worst_emul, worst_exact


def _predict(rg, s, calc, p32, Mt, labels, x, zeta, grad=True, normalize=True):
    import torch

    model = rg.GprModel(calc, Mt, labels, x, zeta=zeta, normalize=normalize)
    ds = rg.DeviceSystem.from_numpy(s)
    e, ea, g = model.predict(ds, torch.tensor(p32, device=calc.device), grad=grad)
    calc.sync()
    return e.cpu().numpy(), ea.cpu().numpy(), (g.cpu().numpy() if g is not None else None)


def _tiny_model():
    s = config_tiny()
    h = osoap.Hypers(**s.hypers)
    p = osoap.power_spectrum(osoap.spherical_expansion(s, h), h, "packed").reshape(s.n_atoms, -1)
    other = config_tiny(seed=9)
    pm = osoap.power_spectrum(osoap.spherical_expansion(other, h, centres=np.arange(40)), h, "packed").reshape(40, -1)
    rng = np.random.default_rng(12)
    return s, h, p.astype(np.float32), pm, other.species[:40], rng.standard_normal(40)


def test_tiny_energies_and_feature_gradient(rg):
    s, h, p32, pm, labels, x = _tiny_model()
    cs = h.species_index(s.species)
    ms = h.species_index(labels)
    Mt = _unit_tf32(pm)
    calc = rg.SoapCalculator(**s.hypers)
    for zeta in (1, 2, 4):
        e, ea, g = _predict(rg, s, calc, p32, Mt, labels, x, zeta)
        p64 = p32.astype(np.float64)
        E_ref = ogpr.energies(p64, cs, pm, ms, x, zeta)
        scale = zeta * np.sum(np.abs(x))
        err = np.max(np.abs(ea - E_ref))
        e_tr = np.max(np.abs(ea - _emulated_energies(p32, cs, Mt, ms, x, zeta, tf32_trunc)))
        e_rn = np.max(np.abs(ea - _emulated_energies(p32, cs, Mt, ms, x, zeta, tf32_nearest)))
        print(f"zeta={zeta} |dE| exact {err / scale:.3e}  vs truncation {e_tr / scale:.3e}  vs nearest {e_rn / scale:.3e}"
              f" (units of zeta sum|x|)")
        assert err <= 2.0 ** -9.4 * scale
        assert min(e_tr, e_rn) <= 1e-5 * scale
        assert abs(e[0] - E_ref.sum()) <= 2.0 ** -9.4 * scale * s.n_atoms
        g_ref = ogpr.grad_p(p64, cs, pm, ms, x, zeta)
        gerr = np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))
        r_emul, r_exact = _grad_checks(g, p32, cs, Mt, ms, x, zeta, pm)
        print(f"zeta={zeta} dE/dp max-relative error {gerr:.3e}; error/allowed: emulated {r_emul:.3f}, exact {r_exact:.3f}")
        assert r_emul <= 1.0 and r_exact <= 1.0


def test_species_buckets_two_passes_odd_features_and_empty_rows(rg):
    """3 species: one with 600 sparse points (two 512-point passes), one with 37, one with none; F odd (4-byte
    copies); a centre with p = 0; two structures."""
    rng = np.random.default_rng(20)
    N, F = 300, 203
    labels3 = [1, 6, 8]
    spe = rng.choice(labels3, size=N).astype(np.int32)
    pos = rng.uniform(0, 20, size=(N, 3))
    s = System(pos, spe, np.stack([np.eye(3) * 20] * 2), np.ones((2, 3), np.int32), np.array([0, 170, N], np.int32),
               dict(r_cut=4.0, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=labels3), "gpr-synthetic")
    p32 = np.abs(rng.normal(size=(N, F))).astype(np.float32)
    p32[5] = 0.0
    n1, n6 = 600, 37
    M = np.abs(rng.normal(size=(n1 + n6, F)))
    mlab = np.array([1] * n1 + [6] * n6, np.int32)
    x = rng.standard_normal(n1 + n6) / 30
    Mt = _unit_tf32(M)
    calc = rg.SoapCalculator(**s.hypers)
    zeta = 3
    e, ea, g = _predict(rg, s, calc, p32, Mt, mlab, x, zeta)
    cs = np.searchsorted(labels3, spe)
    ms = np.searchsorted(labels3, mlab)
    p64 = p32.astype(np.float64)
    E_ref = ogpr.energies(p64, cs, Mt, ms, x, zeta)
    scale = zeta * np.sum(np.abs(x))
    print("two-pass |dE| exact", np.max(np.abs(ea - E_ref)) / scale,
          "vs truncation", np.max(np.abs(ea - _emulated_energies(p32, cs, Mt, ms, x, zeta, tf32_trunc))) / scale)
    assert np.max(np.abs(ea - E_ref)) <= 2.0 ** -9.4 * scale
    assert np.all(ea[spe == 8] == 0.0) and ea[5] == 0.0
    assert np.allclose(e, [ea[:170].astype(np.float64).sum(), ea[170:].astype(np.float64).sum()], rtol=1e-12, atol=1e-12)
    assert np.all(g[spe == 8] == 0.0)
    r_emul, r_exact = _grad_checks(g, p32, cs, Mt, ms, x, zeta, Mt)
    print(f"two-pass dE/dp error/allowed: emulated {r_emul:.3f}, exact {r_exact:.3f}")
    assert r_emul <= 1.0 and r_exact <= 1.0


def test_unnormalised_zeta_one_is_the_linear_model(rg):
    """zeta = 1 without normalisation: E_i = w_{a_i} . p_i with w_a = sum_I x_I M_I, against the GPU linear model."""
    import torch

    s, h, p32, pm, labels, x = _tiny_model()
    Mt = tf32_nearest(pm).astype(np.float64)
    calc = rg.SoapCalculator(**s.hypers)
    e, ea, g = _predict(rg, s, calc, p32, Mt, labels, x, 1, normalize=False)
    w = (x[:, None] * Mt).sum(axis=0, keepdims=True)
    e_lin = calc.linear_energy(rg.DeviceSystem.from_numpy(s), torch.tensor(p32, device=calc.device),
                               torch.tensor(w.astype(np.float32), device=calc.device)).cpu().numpy()
    ref = float(np.sum(p32.astype(np.float64) @ w[0]))
    tol = 2.0 ** -9.4 * float(np.sum((np.abs(p32.astype(np.float64)) @ np.abs(Mt).T) @ np.abs(x)))
    assert abs(e[0] - ref) <= tol and abs(e_lin[0] - ref) <= tol
    # dE/dp = sum_I x_I M_I: the FP32 weights enter the gradient GEMM truncated to TF32
    bound = 2.0 ** -9.4 * (np.abs(x) @ np.abs(Mt))
    assert np.all(np.abs(g - w) <= bound[None, :] + 1e-7)


def test_forces_of_the_gpr_energy_match_the_oracle(rg):
    """The whole path: neighbours, c, p (FP32), the GPR energy and dE/dp, then forces and virial."""
    import torch

    from tests.test_gpu_gradients import _diff_like

    s = _diff_like(n_atoms=200, seed=33)
    h = osoap.Hypers(**s.hypers)
    cs = h.species_index(s.species)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c, p = calc.soap(ds, pairs)
    other = _diff_like(n_atoms=200, seed=34)
    idx, x = gpr_sparse_draws(other.species, h.species, 48, seed=35)
    pm = osoap.power_spectrum(osoap.spherical_expansion(other, h, centres=idx), h, "packed").reshape(idx.size, -1)
    zeta = 2
    model = rg.GprModel(calc, pm, other.species[idx], x, zeta=zeta)
    e, ea, g = model.predict(ds, p, grad=True)
    F, V = calc.gradients(ds, pairs, c, grad_ps=g)
    calc.sync()
    p_ref = osoap.power_spectrum(osoap.spherical_expansion(s, h), h, "packed").reshape(s.n_atoms, -1)
    ms = h.species_index(other.species[idx])
    E_ref = ogpr.energies(p_ref, cs, pm, ms, x, zeta)
    g_ref = ogpr.grad_p(p_ref, cs, pm, ms, x, zeta)
    F_ref, V_ref = osoap.energy_gradients(s, h, None, grad_p=g_ref)
    F, V = F.cpu().numpy(), V.cpu().numpy()
    scale = zeta * np.sum(np.abs(x))
    e_err = np.max(np.abs(ea.cpu().numpy() - E_ref)) / scale
    f_err = np.max(np.abs(F - F_ref)) / np.max(np.abs(F_ref))
    print("E err", e_err, "F err", f_err)
    assert e_err <= 2.0 ** -9.4
    # the gradient kernel on the oracle's own dE/dp (rounded to FP32): the FP32 bar of the linear model
    g32 = g_ref.astype(np.float32)
    F_k, V_k = calc.gradients(ds, pairs, c, grad_ps=torch.tensor(g32, device=calc.device))
    calc.sync()
    F_kr, V_kr = osoap.energy_gradients(s, h, None, grad_p=g32.astype(np.float64))
    assert np.max(np.abs(F_k.cpu().numpy() - F_kr)) <= 1e-4 * np.max(np.abs(F_kr))
    assert np.max(np.abs(V_k.cpu().numpy() - V_kr)) <= 1e-4 * np.max(np.abs(V_kr))
    # end to end against FP64: dE/dp carries the TF32 rounding bounded in the tests above (forces are linear in it)
    assert f_err <= 5e-3
    assert np.max(np.abs(V - V_ref)) <= 5e-3 * np.max(np.abs(V_ref))


def test_model_errors(rg):
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    with pytest.raises(rg.RascalError):
        rg.GprModel(calc, np.ones((2, 5)), [1, 99], [1.0, 1.0])
    with pytest.raises(rg.RascalError):
        rg.GprModel(calc, np.ones((2, 5)), [1, 1], [1.0, 1.0], zeta=0)


def _isolated_system():
    pos = np.array([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0], [9.0, 9.0, 9.0]])
    cells = np.stack([np.eye(3) * 30.0] * 3)
    return System(pos, np.array([14, 14, 14], np.int32), cells, np.array([[1, 1, 1], [0, 0, 0], [1, 1, 1]], np.int32),
                  np.array([0, 1, 1, 3], np.int32), dict(r_cut=5.0, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5,
                                                           species=[14]))


def test_isolated_atoms_empty_structure_and_model_without_points(rg):
    """p = 0 rows (isolated atoms: E = 0, the unnormalised gradient), an empty structure, no atoms at all, and a
    model with no sparse points (E = 0, dE/dp = 0)."""
    import torch

    s = _isolated_system()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    c, p = calc.soap(ds, calc.neighbours(ds))
    F = p.shape[1]
    rng = np.random.default_rng(2)
    M = np.abs(rng.normal(size=(5, F)))
    x = rng.standard_normal(5)
    for zeta in (1, 2):
        model = rg.GprModel(calc, M, [14] * 5, x, zeta=zeta)
        e, ea, g = model.predict(ds, p, grad=True)
        calc.sync()
        p64 = p.double().cpu().numpy()
        assert np.all(p64 == 0.0)
        assert np.all(e.cpu().numpy() == 0.0) and np.all(ea.cpu().numpy() == 0.0)
        g_ref = ogpr.grad_p(p64, np.zeros(3, int), M, np.zeros(5, int), x, zeta)
        # zeta = 1: dE/dp = sum_I x_I M^_I, each term carrying the TF32 rounding of x_I and M^_I (2^-10 + 2^-11);
        # zeta >= 2: exactly 0
        Mh = M / np.linalg.norm(M, axis=1, keepdims=True)
        bound = 2.0 ** -9 * (np.abs(x) @ np.abs(Mh)) + 1e-7
        err = np.abs(g.cpu().numpy() - g_ref)
        print(f"p = 0 rows, zeta {zeta}: max |dg| / bound = {np.max(err / bound[None, :]):.3f}")
        assert np.all(err <= bound[None, :])
    empty = rg.GprModel(calc, np.zeros((0, F)), [], [], zeta=2)
    e, ea, g = empty.predict(ds, p, grad=True)
    calc.sync()
    assert np.all(e.cpu().numpy() == 0.0) and np.all(g.cpu().numpy() == 0.0)
    # no atoms at all
    s0 = System(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3)[None] * 10.0, np.ones((1, 3), np.int32),
                np.array([0, 0], np.int32), s.hypers)
    ds0 = rg.DeviceSystem.from_numpy(s0)
    e0, _, g0 = rg.GprModel(calc, M, [14] * 5, x).predict(ds0, torch.zeros((0, F), device=calc.device), grad=True)
    calc.sync()
    assert e0.shape == (1,) and float(e0.cpu()[0]) == 0.0 and g0.shape == (0, F)


def test_batch_full_size_sampled(rg):
    """The bench's configuration: batch workload, fused FP32 p, 512 sparse points per species (from the oracle's p of
    the drawn atoms), zeta 2; energies and dE/dp of sampled centres against FP64 on the oracle's p."""
    from synth import config_batch

    s = config_batch()
    h = osoap.Hypers(**s.hypers)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c, p = calc.soap(ds, pairs)
    idx, x = gpr_sparse_draws(s.species, h.species, 512, seed=31)
    pm = osoap.power_spectrum(osoap.spherical_expansion(s, h, centres=idx), h, "packed").reshape(idx.size, -1)
    model = rg.GprModel(calc, pm, s.species[idx], x, zeta=2)
    e, ea, g = model.predict(ds, p, grad=True)
    calc.sync()
    rng = np.random.default_rng(3)
    centres = np.concatenate([[0, s.n_atoms - 1], rng.choice(s.n_atoms, 14, replace=False)])
    p_ref = osoap.power_spectrum(osoap.spherical_expansion(s, h, centres=centres), h, "packed").reshape(centres.size, -1)
    a = h.species_index(s.species)
    ms = h.species_index(s.species[idx])
    E_ref = ogpr.energies(p_ref, a[centres], pm, ms, x, 2)
    g_ref = ogpr.grad_p(p_ref, a[centres], pm, ms, x, 2)
    scale = 2 * np.sum(np.abs(x[ms == a[0]]))  # |x| of one species' points bounds that species' energies
    e_err = np.max(np.abs(ea.cpu().numpy()[centres] - E_ref))
    g_gpu = g[_on_device(centres, g)].cpu().numpy()
    g_err = np.max(np.abs(g_gpu - g_ref)) / np.max(np.abs(g_ref))
    print(f"batch: |dE| {e_err:.3e} (bound unit {scale:.3e}), dE/dp max-relative {g_err:.3e}")
    assert e_err <= 2.0 ** -9 * 2 * np.sum(np.abs(x))
    assert g_err <= 1e-2
    assert np.isfinite(e.cpu().numpy()).all()


def _on_device(idx, like):
    import torch

    return torch.as_tensor(idx, device=like.device)
