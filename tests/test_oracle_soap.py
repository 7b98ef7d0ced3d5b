"""Pins of the oracle's coefficients, power spectrum, linear energy and gradients."""
from math import pi, sqrt
import os

import numpy as np
import pytest

from oracle import radial, soap, ylm
from synth import System, config_tiny, linear_weights, small_cell_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _two_atoms(d, species=(14, 14), L=30.0):
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0]]) + np.array([[0, 0, 0], d])
    return System(pos, np.array(species, np.int32), (np.eye(3) * L)[None], np.ones((1, 3), np.int32),
                  np.array([0, 2], np.int32))


def _rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


H1 = soap.Hypers(r_cut=5.0, sigma=0.5, n_max=6, l_max=5, species=[14])
H2 = soap.Hypers(r_cut=5.0, sigma=0.5, n_max=4, l_max=4, species=[1, 6])


def test_cutoff_function_values():
    rc, w = 5.0, 0.5
    assert soap.cutoff(4.5, rc, w) == 1.0 and soap.cutoff(5.0, rc, w) == 0.0
    assert abs(soap.cutoff(4.75, rc, w) - 0.5) < 1e-15
    f, df = soap.cutoff(np.array([4.6, 4.9]), rc, w, derivative=True)
    h = 1e-6
    assert np.allclose(df, (soap.cutoff(np.array([4.6, 4.9]) + h, rc, w) - soap.cutoff(np.array([4.6, 4.9]) - h, rc, w)) / (2 * h))


def test_single_neighbour_coefficients_and_power_spectrum_closed_form():
    d = np.array([1.1, -2.0, 0.7])
    s = _two_atoms(d)
    c = soap.spherical_expansion(s, H1)
    r = np.linalg.norm(d)
    f = soap.cutoff(r, 5.0, 0.5)
    I = radial.integrals(np.array([r]), 5.0, 0.5, 6, 5)[0]
    Y = ylm.real_ylm(d[None], 5)[0]
    lidx = np.array([l for l in range(6) for _ in range(2 * l + 1)])
    assert np.allclose(c[0, 0], f * I[:, lidx] * Y[None, :], atol=1e-15)
    # single neighbour: p_{n1 n2 l} = f^2 I_n1l I_n2l sqrt(2l+1)/(4 pi), independent of direction
    p = soap.power_spectrum(c, H1, "full")
    for l in range(6):
        ref = f * f * np.outer(I[:, l], I[:, l]) * sqrt(2 * l + 1) / (4 * pi)
        assert np.allclose(p[0, l], ref, atol=1e-14)


def test_power_spectrum_matches_ylm_free_bruteforce():
    s = config_tiny()
    h = soap.Hypers(**dict(s.hypers, n_max=5, l_max=6))
    for centre in [0, 17, 63]:
        c = soap.spherical_expansion(s, h, centres=[centre])
        p = soap.power_spectrum(c, h, "full")[0]
        ref = soap.power_spectrum_bruteforce(s, h, centre)
        assert np.allclose(p, ref, atol=1e-12 * np.max(np.abs(ref)))


def test_power_spectrum_invariances_and_symmetry():
    s = small_cell_system(seed=5, n_atoms=7, L=5.5, hypers=dict(r_cut=5.0, sigma=0.5, n_max=4, l_max=4, smooth_width=0.5, species=[1, 6]))
    h = soap.Hypers(**s.hypers)
    p0 = soap.power_spectrum(soap.spherical_expansion(s, h), h, "full")
    assert np.allclose(p0, np.transpose(p0, (0, 1, 3, 2)), atol=1e-14)
    R = _rotation(3)
    rot = System(s.positions @ R.T, s.species, s.cells @ R.T, s.pbc, s.struct_offsets, s.hypers)
    assert np.allclose(soap.power_spectrum(soap.spherical_expansion(rot, h), h, "full"), p0, atol=1e-11)
    inv = System(-s.positions, s.species, -s.cells, s.pbc, s.struct_offsets, s.hypers)
    assert np.allclose(soap.power_spectrum(soap.spherical_expansion(inv, h), h, "full"), p0, atol=1e-11)
    tr = System(s.positions + np.array([0.3, -1.7, 2.2]), s.species, s.cells, s.pbc, s.struct_offsets, s.hypers)
    assert np.allclose(soap.power_spectrum(soap.spherical_expansion(tr, h), h, "full"), p0, atol=1e-11)
    perm = np.random.default_rng(0).permutation(s.n_atoms)
    pm = System(s.positions[perm], s.species[perm], s.cells, s.pbc, s.struct_offsets, s.hypers)
    assert np.allclose(soap.power_spectrum(soap.spherical_expansion(pm, h), h, "full"), p0[perm], atol=1e-11)


def test_coefficients_rotate_covariantly_per_l():
    # c_l transforms with an orthogonal (2l+1)x(2l+1) matrix: the per-l Gram C_l C_l^T is invariant, and the
    # linear map between rotated and original c_l is orthogonal
    s = config_tiny()
    h = soap.Hypers(**dict(s.hypers, n_max=4, l_max=3))
    R = _rotation(7)
    rot = System(s.positions @ R.T, s.species, s.cells @ R.T, s.pbc, s.struct_offsets, s.hypers)
    c0 = soap.spherical_expansion(s, h, centres=list(range(10)))
    c1 = soap.spherical_expansion(rot, h, centres=list(range(10)))
    for l in range(1, 4):
        sl = slice(l * l, (l + 1) * (l + 1))
        A = c0[:, 0, :, sl].reshape(-1, 2 * l + 1)
        B = c1[:, 0, :, sl].reshape(-1, 2 * l + 1)
        D, *_ = np.linalg.lstsq(A, B, rcond=None)
        assert np.allclose(A @ D, B, atol=1e-10)
        assert np.allclose(D.T @ D, np.eye(2 * l + 1), atol=1e-8)


def test_packed_feature_counts_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "feature_counts.txt")) if l.strip() and not l.startswith("#")]
    for r in rows:
        S, n, lm, count = map(int, r[:4])
        h = soap.Hypers(r_cut=5.0, sigma=0.5, n_max=n, l_max=lm, species=list(range(1, S + 1)))
        assert h.n_features("packed") == count


def test_packed_layout_is_upper_triangle_of_full():
    s = config_tiny()
    h = soap.Hypers(**dict(s.hypers, n_max=3, l_max=2))
    c = soap.spherical_expansion(s, h, centres=[0, 5])
    full = soap.power_spectrum(c, h, "full")
    packed = soap.power_spectrum(c, h, "packed")
    Q = h.q
    k = 0
    for q1 in range(Q):
        for q2 in range(q1, Q):
            assert np.allclose(packed[:, :, k], full[:, :, q1, q2])
            k += 1


def _fd_forces(s, h, w, atoms, step=1e-4):
    out = np.zeros((len(atoms), 3))
    for t, a in enumerate(atoms):
        for k in range(3):
            sp = System(s.positions.copy(), s.species, s.cells, s.pbc, s.struct_offsets, s.hypers)
            sm = System(s.positions.copy(), s.species, s.cells, s.pbc, s.struct_offsets, s.hypers)
            sp.positions[a, k] += step
            sm.positions[a, k] -= step
            out[t, k] = -(soap.total_energy(sp, h, w) - soap.total_energy(sm, h, w)) / (2 * step)
    return out


def test_forces_and_virial_against_finite_differences():
    s = small_cell_system(seed=9, n_atoms=6, L=5.2, hypers=dict(r_cut=4.5, sigma=0.45, n_max=4, l_max=3, smooth_width=0.5, species=[1, 6]))
    h = soap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=4)
    F, V = soap.energy_gradients(s, h, w)
    fd = _fd_forces(s, h, w, [0, 3, 5])
    assert np.allclose(F[[0, 3, 5]], fd, atol=1e-6 * max(1.0, np.max(np.abs(fd))))
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-10 * np.max(np.abs(F)))
    assert np.allclose(V[0], V[0].T, atol=1e-9 * np.max(np.abs(V)))
    # strain derivative: r -> (1 + eta) r for positions and cell vectors
    eps = 1e-6
    fdV = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            E = []
            for sg in (1, -1):
                D = np.eye(3)
                D[a, b] += sg * eps
                st = System(s.positions @ D.T, s.species, s.cells @ D.T, s.pbc, s.struct_offsets, s.hypers)
                E.append(soap.total_energy(st, h, w))
            fdV[a, b] = (E[0] - E[1]) / (2 * eps)
    assert np.allclose(V[0], fdV, atol=1e-5 * max(1.0, np.max(np.abs(fdV))))


def test_gradients_of_a_centre_subset_add_up_to_the_whole():
    # E is a sum over centres, so the gradients of the energy terms of a partition of the centres add up to the
    # gradients of E; the partial sums are what the timed CPU samples compute
    s = small_cell_system(seed=5, n_atoms=7, L=5.6, hypers=dict(r_cut=4.5, sigma=0.45, n_max=3, l_max=3, smooth_width=0.5, species=[1, 6]))
    h = soap.Hypers(**s.hypers)
    w = linear_weights(h.n_species, h.n_features("packed"), seed=6)
    F, V = soap.energy_gradients(s, h, w)
    Fa, Va = soap.energy_gradients(s, h, w, centres=[0, 2, 5])
    Fb, Vb = soap.energy_gradients(s, h, w, centres=[6, 1, 3, 4])
    assert np.allclose(Fa + Fb, F, atol=1e-12 * np.max(np.abs(F)))
    assert np.allclose(Va + Vb, V, atol=1e-12 * np.max(np.abs(V)))
    assert not np.allclose(Fa, F)


def test_self_images_give_no_force_but_virial():
    # one atom in a cell narrower than r_cut: the environment holds only images of the atom itself
    cell = np.array([[3.1, 0.0, 0.0], [0.4, 3.3, 0.0], [0.2, -0.5, 3.6]])
    s = System(np.array([[0.3, 0.2, 0.1]]), np.array([14], np.int32), cell[None], np.ones((1, 3), np.int32), np.array([0, 1], np.int32))
    h = soap.Hypers(r_cut=5.0, sigma=0.5, n_max=3, l_max=2, species=[14])
    w = linear_weights(1, h.n_features("packed"), seed=2)
    F, V = soap.energy_gradients(s, h, w)
    assert np.all(F == 0.0)
    assert np.max(np.abs(V)) > 1e-3
    assert np.allclose(_fd_forces(s, h, w, [0]), 0.0, atol=1e-8)


def test_spline_mode_matches_exact_coefficients():
    s = config_tiny()
    h = soap.Hypers(**dict(s.hypers, n_max=4, l_max=3))
    sp = radial.RadialSpline(h.r_cut, h.sigma, h.n_max, h.l_max, accuracy=1e-8)
    c_ex = soap.spherical_expansion(s, h, centres=[0, 1, 2])
    c_sp = soap.spherical_expansion(s, h, centres=[0, 1, 2], radial_fn=lambda r, d: sp(r, d))
    assert np.max(np.abs(c_ex - c_sp)) < 40 * 1e-8


def test_include_center_adds_l0_term_only():
    s = config_tiny()
    h0 = soap.Hypers(**dict(s.hypers, n_max=3, l_max=2))
    h1 = soap.Hypers(**dict(s.hypers, n_max=3, l_max=2, include_center=True))
    d = soap.spherical_expansion(s, h1, centres=[4]) - soap.spherical_expansion(s, h0, centres=[4])
    assert np.all(d[..., 1:] == 0.0)
    I0 = radial.integrals(np.array([0.0]), h0.r_cut, h0.sigma, 3, 2)[0][:, 0]
    assert np.allclose(d[0, 0, :, 0], I0 / (2 * sqrt(pi)))


def test_three_species_power_spectrum_matches_ylm_free_bruteforce():
    # species channel of Eq. spherical_expansion_coefficients_gaussians: neighbour j adds only to block a_j, with
    # blocks ordered by the sorted labels (the labels are given unsorted); the brute force assigns each neighbour's
    # radial row by its own species and never forms c, so a term routed to the wrong block (e.g. the centre's
    # species) changes the off-diagonal species blocks of p and fails here
    hyp = dict(r_cut=4.5, sigma=0.45, n_max=3, l_max=4, smooth_width=0.5, species=[8, 1, 6])
    s = small_cell_system(seed=17, n_atoms=9, L=4.6, hypers=hyp)
    assert set(np.unique(s.species)) == {1, 6, 8}
    h = soap.Hypers(**s.hypers)
    for centre in range(s.n_atoms):
        p = soap.power_spectrum(soap.spherical_expansion(s, h, centres=[centre]), h, "full")[0]
        ref = soap.power_spectrum_bruteforce(s, h, centre)
        assert np.max(np.abs(ref)) > 0.0
        assert np.allclose(p, ref, rtol=0.0, atol=1e-12 * np.max(np.abs(ref))), centre


def test_two_species_single_neighbour_fills_only_its_own_block():
    # one neighbour of label 8 around a centre of label 1, hypers listing the labels unsorted: c is non-zero only in
    # block a_j = 2 (sorted labels 1, 6, 8), and p only in the (a_j, a_j) block, where it takes the closed form
    # f^2 I_n1l I_n2l sqrt(2l+1)/(4 pi) of a single neighbour
    h = soap.Hypers(r_cut=5.0, sigma=0.5, n_max=4, l_max=3, species=[8, 1, 6])
    d = np.array([0.4, -1.9, 1.3])
    s = _two_atoms(d, species=(1, 8))
    c = soap.spherical_expansion(s, h, centres=[0])[0]            # [S, n, lm]
    r = np.linalg.norm(d)
    f = soap.cutoff(r, 5.0, 0.5)
    I = radial.integrals(np.array([r]), 5.0, 0.5, 4, 3)[0]
    Y = ylm.real_ylm(d[None], 3)[0]
    lidx = np.array([l for l in range(4) for _ in range(2 * l + 1)])
    assert np.all(c[0] == 0.0) and np.all(c[1] == 0.0)
    assert np.allclose(c[2], f * I[:, lidx] * Y[None, :], atol=1e-15)
    p = soap.power_spectrum(c[None], h, "full")[0]                 # [l, Q, Q]
    n = 4
    for l in range(4):
        blk = np.zeros((12, 12))
        blk[2 * n:3 * n, 2 * n:3 * n] = f * f * np.outer(I[:, l], I[:, l]) * sqrt(2 * l + 1) / (4 * pi)
        assert np.allclose(p[l], blk, atol=1e-14)
    # the centre of label 8 seen from the other side: its neighbour (label 1) fills block 0 only
    c1 = soap.spherical_expansion(s, h, centres=[1])[0]
    assert np.any(c1[0] != 0.0) and np.all(c1[1] == 0.0) and np.all(c1[2] == 0.0)
