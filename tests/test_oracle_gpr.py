"""Pins of the oracle's sparse GPR model (Eq. sparse-gp with the polynomial kernel) against closed forms, the
linear model it reduces to, invariances and central differences."""
import numpy as np
import pytest

from oracle import gpr, soap


def _model(rng, n_centres=7, F=12, n_sparse=9, n_species=2):
    p = np.abs(rng.normal(size=(n_centres, F))) + 0.1 * rng.normal(size=(n_centres, F))
    cs = rng.integers(0, n_species, n_centres)
    M = np.abs(rng.normal(size=(n_sparse, F)))
    ms = rng.integers(0, n_species, n_sparse)
    x = rng.normal(size=n_sparse)
    return p, cs, M, ms, x


def test_zeta_one_unnormalised_is_the_linear_model():
    rng = np.random.default_rng(1)
    p, cs, M, ms, x = _model(rng)
    w = np.stack([(x[ms == s, None] * M[ms == s]).sum(axis=0) for s in range(2)])
    E_lin = soap.linear_energy(p, cs, w)[1]
    assert np.allclose(gpr.energies(p, cs, M, ms, x, 1, normalize=False), E_lin, rtol=1e-13, atol=1e-13)
    assert np.allclose(gpr.grad_p(p, cs, M, ms, x, 1, normalize=False), w[cs], rtol=1e-13, atol=1e-13)


def test_self_similarity_and_opposite_direction():
    rng = np.random.default_rng(2)
    p = rng.normal(size=(3, 10))
    cs = np.array([0, 0, 0])
    for zeta in (1, 2, 3, 4):
        # the only sparse point is a positive multiple of centre 1, another is its negative
        M = np.stack([3.7 * p[1], -0.5 * p[1]])
        E = gpr.energies(p, cs, M, np.array([0, 0]), np.array([0.25, 2.0]), zeta)
        assert np.isclose(E[1], 0.25 + 2.0 * (-1) ** zeta, rtol=1e-14)


def test_normalised_model_is_scale_invariant_and_its_gradient_is_orthogonal_to_p():
    rng = np.random.default_rng(3)
    p, cs, M, ms, x = _model(rng)
    for zeta in (2, 3):
        E = gpr.energies(p, cs, M, ms, x, zeta)
        lam = rng.uniform(0.1, 10.0, size=(p.shape[0], 1))
        assert np.allclose(gpr.energies(lam * p, cs, 2.5 * M, ms, x, zeta), E, rtol=1e-12)
        g = gpr.grad_p(p, cs, M, ms, x, zeta)
        assert np.allclose(np.sum(g * p, axis=1), 0.0, atol=1e-12 * np.max(np.abs(g)))
        # Euler: the unnormalised kernel is homogeneous of degree zeta in p, so g . p = zeta E
        gu = gpr.grad_p(p, cs, M, ms, x, zeta, normalize=False)
        Eu = gpr.energies(p, cs, M, ms, x, zeta, normalize=False)
        assert np.allclose(np.sum(gu * p, axis=1), zeta * Eu, rtol=1e-12)


@pytest.mark.parametrize("zeta,normalize", [(2, True), (3, True), (4, True), (2, False), (3, False)])
def test_gradient_against_central_differences(zeta, normalize):
    rng = np.random.default_rng(10 + zeta)
    p, cs, M, ms, x = _model(rng)
    g = gpr.grad_p(p, cs, M, ms, x, zeta, normalize)
    h = 1e-6
    for i, q in [(0, 0), (2, 5), (4, 11), (6, 3)]:
        pp, pm = p.copy(), p.copy()
        pp[i, q] += h
        pm[i, q] -= h
        fd = (gpr.energies(pp, cs, M, ms, x, zeta, normalize)[i] - gpr.energies(pm, cs, M, ms, x, zeta, normalize)[i]) / (2 * h)
        assert np.isclose(g[i, q], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(g)))


def test_centres_without_sparse_points_of_their_species_have_no_energy():
    rng = np.random.default_rng(5)
    p, cs, M, ms, x = _model(rng, n_species=3)
    ms = np.where(ms == 2, 0, ms)  # no sparse point of species 2
    E = gpr.energies(p, cs, M, ms, x, 2)
    g = gpr.grad_p(p, cs, M, ms, x, 2)
    assert np.all(E[cs == 2] == 0.0) and np.all(g[cs == 2] == 0.0)


def test_forces_of_the_gpr_energy_against_central_differences_of_positions():
    from synth import small_cell_system

    s = small_cell_system(seed=41, n_atoms=6, L=4.6, hypers=dict(r_cut=4.0, sigma=0.5, n_max=4, l_max=3,
                                                                 smooth_width=0.6, species=[1, 8]))
    h = soap.Hypers(**s.hypers)
    a = h.species_index(s.species)
    rng = np.random.default_rng(6)
    # sparse points: the FP64 power spectra of the same kind of system with other positions
    other = small_cell_system(seed=42, n_atoms=6, L=4.6, hypers=s.hypers)
    M = soap.power_spectrum(soap.spherical_expansion(other, h), h, "packed").reshape(6, -1)
    ms = h.species_index(other.species)
    x = rng.normal(size=M.shape[0])
    zeta = 3

    def total(pos):
        s.positions = pos
        p = soap.power_spectrum(soap.spherical_expansion(s, h), h, "packed").reshape(s.n_atoms, -1)
        return gpr.energies(p, a, M, ms, x, zeta).sum(), p

    pos0 = s.positions.copy()
    _, p0 = total(pos0)
    F, _ = soap.energy_gradients(s, h, None, grad_p=gpr.grad_p(p0, a, M, ms, x, zeta))
    hstep = 1e-5
    for atom, ax in [(0, 0), (3, 2), (5, 1)]:
        dp, dm = pos0.copy(), pos0.copy()
        dp[atom, ax] += hstep
        dm[atom, ax] -= hstep
        fd = -(total(dp)[0] - total(dm)[0]) / (2 * hstep)
        assert np.isclose(F[atom, ax], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(F)))
    s.positions = pos0
