"""GPU backward pass (forces, virial, autograd) against the FP64 oracle's analytic gradients and finite differences.

Tolerance (FP32 path): max |F_gpu - F_oracle| / max |F_oracle| <= 1e-4, the same for the virial.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import soap as osoap  # noqa: E402
from synth import System, config_diff, linear_weights, random_cell_atoms, small_cell_system  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _diff_like(n_atoms=400, seed=31):
    """The differentiation workload's hypers and density on a smaller cell (2 species 1:1, 0.05 atoms/A^3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (n_atoms / 0.05) ** (1 / 3)
    pos = random_cell_atoms(n_atoms, np.eye(3) * L, 1.8, rng)
    spe = np.array([1, 6] * (n_atoms // 2), np.int32)
    rng.shuffle(spe)
    h = dict(config_diff().hypers)
    return System(pos, spe, (np.eye(3) * L)[None], np.ones((1, 3), np.int32), np.array([0, n_atoms], np.int32), h, "diff-small")


def _gpu_forces(rg, s, w):
    import torch

    from paper_2101_08814_gb300.autograd import LinearSoapEnergy

    calc = rg.SoapCalculator(**s.hypers)
    model = LinearSoapEnergy(calc, torch.tensor(w, dtype=torch.float32))
    ds = rg.DeviceSystem.from_numpy(s)
    e, f, v = model(ds)
    calc.sync()
    return calc, ds, model, e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy()


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_forces_and_virial_match_oracle(rg):
    s = _diff_like()
    h = osoap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    _, _, _, e, f, v = _gpu_forces(rg, s, w)
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    E_ref = osoap.total_energy(s, h, w)
    assert abs(e[0] - E_ref) <= 1e-5 * abs(E_ref)
    assert _rel(f, F_ref) <= TOL
    assert _rel(v, V_ref) <= TOL
    assert np.allclose(f.sum(axis=0), 0.0, atol=1e-4 * np.max(np.abs(f)))
    assert np.allclose(v[0], v[0].T, atol=1e-4 * np.max(np.abs(v)))


def test_self_images_small_cell(rg):
    s = small_cell_system(seed=9, n_atoms=6, L=5.2, hypers=dict(r_cut=4.5, sigma=0.45, n_max=4, l_max=3, smooth_width=0.5,
                                                               species=[1, 6]))
    h = osoap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    _, _, _, _, f, v = _gpu_forces(rg, s, w)
    F_ref, V_ref = osoap.energy_gradients(s, h, w)
    assert _rel(f, F_ref) <= TOL
    assert _rel(v, V_ref) <= TOL


def test_autograd_matches_forces_and_grad_ps_mode(rg):
    import torch

    from paper_2101_08814_gb300.autograd import power_spectrum

    s = _diff_like(200, seed=5)
    h = osoap.Hypers(**s.hypers)
    w = torch.tensor(linear_weights(h.n_species, h.n_features("packed"), seed=4), dtype=torch.float32, device="cuda")
    calc, ds, model, e, f, v = _gpu_forces(rg, s, w.cpu().numpy())
    pos = ds.positions.clone().requires_grad_(True)
    p = power_spectrum(pos, calc, ds)
    a = torch.as_tensor(h.species_index(s.species), device="cuda")
    E = (p.double() * w[a].double()).sum()
    (g,) = torch.autograd.grad(E, pos)
    assert abs(E.item() - e[0]) <= 1e-6 * abs(e[0])
    assert np.max(np.abs(-g.cpu().numpy() - f)) <= 1e-5 * np.max(np.abs(f))


def test_central_finite_differences_of_gpu_energy(rg):
    # h = 1e-4 A on the GPU energy (FP32 features, FP64 energy sum): FP32 rounding of the few centres that see the
    # displaced atom sets a noise floor of about 1e-7 |E_local| / h, so this is a 2 % check
    import torch

    s = _diff_like(300, seed=8)
    h = osoap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    calc, ds, model, e, f, v = _gpu_forces(rg, s, w)
    step = 1e-4
    for atom in (0, 137):
        for k in range(3):
            out = []
            for sg in (1, -1):
                pos = ds.positions.clone()
                pos[atom, k] += sg * step
                d2 = rg.DeviceSystem(pos, ds.species, ds.cells, ds.pbc, ds.struct_offsets)
                out.append(model(d2, forces=False)[0].sum().item())
            fd = -(out[0] - out[1]) / (2 * step)
            assert abs(fd - f[atom, k]) <= 2e-2 * np.max(np.abs(f)), (atom, k, fd, f[atom, k])


def test_full_size_differentiation_workload_properties(rg):
    s = config_diff()
    h = osoap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    _, _, _, e, f, v = _gpu_forces(rg, s, w)
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(v))
    assert np.allclose(f.sum(axis=0), 0.0, atol=1e-4 * np.max(np.abs(f)) * np.sqrt(s.n_atoms))
    assert np.allclose(v[0], v[0].T, atol=1e-4 * np.max(np.abs(v)))
    assert abs(np.sum(f * s.positions)) > 0.0


def _oracle_pair_terms(d, hyp, derivative):
    """The oracle's f_cut I^o_nl Y_lm of one pair vector d (and its gradient d/dd_x): [n, lm] or [3, n, lm]."""
    from oracle import radial as oradial
    from oracle import ylm as oylm

    r = np.linalg.norm(d, axis=1)
    f, df = osoap.cutoff(r, hyp["r_cut"], hyp["smooth_width"], derivative=True)
    I, dI = oradial.integrals(r, hyp["r_cut"], hyp["sigma"], hyp["n_max"], hyp["l_max"], derivative=True)
    Y, dY = oylm.real_ylm(d, hyp["l_max"], gradient=True)               # [P, lm], [P, lm, 3]
    lidx = np.array([l for l in range(hyp["l_max"] + 1) for _ in range(2 * l + 1)])
    R = f[:, None, None] * I[:, :, lidx]                                  # [P, n, lm]
    if not derivative:
        return R * Y[:, None, :]
    dR = df[:, None, None] * I[:, :, lidx] + f[:, None, None] * dI[:, :, lidx]
    u = d / r[:, None]
    return (np.einsum("pnk,pk,px->pxnk", dR, Y, u) + np.einsum("pnk,pkx->pxnk", R, dY))


def test_debug_pair_gradients_match_oracle(rg):
    # the per-pair feature gradient written out (Appendix B): d/dr_ji of f_cut I^o_nl Y_lm, against the oracle's
    # analytic gradient, and the oracle's analytic gradient against its own central differences; pairs of the tiny
    # workload plus pairs near the cutoff's smooth zone and on the +z / -z axis (the Y_lm pole)
    import torch

    from synth import config_tiny

    s = config_tiny()
    hyp = dict(s.hypers)
    calc = rg.SoapCalculator(**hyp)
    pl = calc.neighbours(rg.DeviceSystem.from_numpy(s))
    rij = pl.rij[:300].cpu().numpy().astype(np.float64)
    extra = np.array([[0.3, -0.2, 4.8], [0.0, 0.0, 2.1], [0.0, 0.0, -3.3], [1e-3, 0.0, 4.0], [4.6, 0.9, -0.5]])
    d = np.concatenate([rij[:, :3], extra])
    d32 = d.astype(np.float32)
    rows = np.concatenate([d32, np.linalg.norm(d32.astype(np.float64), axis=1).astype(np.float32)[:, None]], axis=1)
    got = calc.debug_pair_gradients(torch.tensor(rows, device="cuda")).cpu().numpy().astype(np.float64)
    ref = _oracle_pair_terms(d32.astype(np.float64), hyp, True)
    # the FP32 spline's absolute error enters every pair's block alike: pairs inside the smooth zone of the cutoff
    # (f_cut = 1) are held to 1e-5 of their own block's maximum; near r_cut, where f_cut and the whole block tend to
    # zero, the error is held to 1e-5 of the largest pair term of the set instead (the scale that c and the forces see)
    absd = np.abs(got - ref).reshape(len(d), -1)
    blk = np.max(np.abs(ref).reshape(len(d), -1), axis=1)
    r = np.linalg.norm(d32.astype(np.float64), axis=1)
    inner = r <= hyp["r_cut"] - hyp["smooth_width"]
    err_in = np.max(absd[inner], axis=1) / blk[inner]
    err_all = np.max(absd) / np.max(blk)
    print(f"per-pair gradient: block error {err_in.max():.2e} ({inner.sum()} pairs with f_cut = 1), "
          f"{err_all:.2e} of the largest term over all {len(d)} pairs")
    assert err_in.max() <= 1e-5 and err_all <= 1e-5, (err_in.max(), err_all)
    # the oracle's analytic pair gradient against central differences of its own pair term (h = 1e-5 A)
    h = 1e-5
    for x in range(3):
        e = np.zeros(3)
        e[x] = h
        fd = (_oracle_pair_terms(d + e, hyp, False) - _oracle_pair_terms(d - e, hyp, False)) / (2 * h)
        an = _oracle_pair_terms(d, hyp, True)[:, x]
        assert np.max(np.abs(fd - an)) <= 1e-7 * max(1.0, np.max(np.abs(an)))
