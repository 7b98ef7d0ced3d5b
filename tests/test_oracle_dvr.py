"""Pins of the oracle's DVR radial basis (Eq. rad-int-dvr) against closed forms and quadrature."""
import numpy as np
import pytest

from oracle import dvr, ylm

A = 1.0 / (2 * 0.5 ** 2)  # a = 1/(2 sigma^2) at sigma = 0.5


def test_scaled_bessel_closed_forms_and_library():
    z = np.array([0.3, 2.0, 17.0, 150.0])
    e = dvr.scaled_bessel_i(3, z)
    i0 = np.sinh(z) / z
    i1 = (z * np.cosh(z) - np.sinh(z)) / z ** 2
    i2 = ((z * z + 3) * np.sinh(z) - 3 * z * np.cosh(z)) / z ** 3
    for l, il in enumerate([i0, i1, i2]):
        ok = z < 50  # the unscaled closed forms overflow beyond
        assert np.allclose(e[ok, l], np.exp(-z[ok]) * il[ok], rtol=1e-12, atol=0)
    from scipy import special

    zz = np.array([0.01, 0.5, 3.0, 30.0])
    for l in range(4):
        assert np.allclose(dvr.scaled_bessel_i(3, zz)[:, l], np.exp(-zz) * special.spherical_in(l, zz), rtol=1e-12)
    # small-argument series against the library form on both sides of its switch
    zs = np.array([0.9e-4, 1.1e-4])
    e_s = dvr.scaled_bessel_i(3, zs)
    for l in range(4):
        assert np.allclose(e_s[:, l], np.exp(-zs) * special.spherical_in(l, zs), rtol=1e-10, atol=1e-300)


def test_gauss_legendre_nodes():
    x, w = dvr.nodes(5.0, 0.5, 6)
    assert np.isclose(w.sum(), 6.5) and np.all((x > 0) & (x < 6.5))
    for k in range(2 * 6):  # exact for polynomials of degree 2 n_max - 1
        assert np.isclose(np.sum(w * x ** k), 6.5 ** (k + 1) / (k + 1), rtol=1e-12)


def _angular_projection(xv, rv, l_max, n_t=64, n_p=128):
    """int dOmega_x Y_lm(x^) exp(-a |x - r|^2) over directions of x at fixed |x|, by quadrature."""
    t, wt = np.polynomial.legendre.leggauss(n_t)
    phi = (np.arange(n_p) + 0.5) * 2 * np.pi / n_p
    ct, ph = np.meshgrid(t, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    weights = (wt[:, None] * np.full(n_p, 2 * np.pi / n_p)[None, :]).reshape(-1)
    Y = ylm.real_ylm(dirs, l_max)                                  # [K, (l_max+1)^2]
    f = np.exp(-A * np.sum((xv * dirs - rv) ** 2, axis=1))
    return np.einsum("k,k,kj->j", weights, f, Y)


def test_angular_identity_fixes_prefactor_exponent_and_bessel():
    rng = np.random.default_rng(4)
    l_max = 4
    for _ in range(3):
        x = rng.uniform(0.3, 6.0)
        rv = rng.normal(size=3)
        rv *= rng.uniform(0.2, 4.5) / np.linalg.norm(rv)
        r = np.linalg.norm(rv)
        proj = _angular_projection(x, rv, l_max)
        e = dvr.scaled_bessel_i(l_max, 2 * A * x * r)[0]
        Yr = ylm.real_ylm(rv[None, :], l_max)[0]
        for l in range(l_max + 1):
            sl = slice(l * l, (l + 1) ** 2)
            expect = 4 * np.pi * np.exp(-A * (x - r) ** 2) * e[l] * Yr[sl]
            assert np.allclose(proj[sl], expect, atol=1e-10 * max(1.0, np.max(np.abs(expect))))


def test_dvr_integral_is_the_node_projection():
    r_cut, sigma, n_max, l_max = 5.0, 0.5, 5, 3
    x, w = dvr.nodes(r_cut, sigma, n_max)
    I = dvr.integrals(np.array([0.7, 2.3, 4.1]), r_cut, sigma, n_max, l_max)
    rng = np.random.default_rng(8)
    for k, r in enumerate([0.7, 2.3, 4.1]):
        u = rng.normal(size=3)
        rv = r * u / np.linalg.norm(u)
        Yr = ylm.real_ylm(rv[None, :], l_max)[0]
        for n in (0, 2, 4):
            proj = _angular_projection(x[n], rv, l_max)
            for l in range(l_max + 1):
                m0 = l * l + l  # the m = 0 component carries Y_l0(r^), nonzero for a generic direction
                assert np.isclose(x[n] * np.sqrt(w[n]) * proj[m0], I[k, n, l] * Yr[m0],
                                  rtol=1e-9, atol=1e-12 * np.max(np.abs(I[k, n])))


def test_derivative_against_central_differences_and_r0():
    r = np.array([0.0, 0.4, 1.7, 3.3, 4.8])
    I, dI = dvr.integrals(r, 5.0, 0.5, 4, 4, derivative=True)
    h = 1e-6
    for k in range(1, r.size):
        fd = (dvr.integrals(r[k] + h, 5.0, 0.5, 4, 4) - dvr.integrals(r[k] - h, 5.0, 0.5, 4, 4))[0] / (2 * h)
        assert np.allclose(dI[k], fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(I[k])))
    assert np.all(I[0, :, 1:] == 0.0)  # only l = 0 survives at r = 0
    h0 = 1e-4  # one-sided second-order difference at r = 0
    fd0 = (-3 * I[0] + 4 * dvr.integrals(h0, 5.0, 0.5, 4, 4)[0] - dvr.integrals(2 * h0, 5.0, 0.5, 4, 4)[0]) / (2 * h0)
    assert np.allclose(dI[0], fd0, rtol=1e-6, atol=1e-7 * np.max(np.abs(dI[0])))


def test_dvr_basis_power_spectrum_matches_ylm_free_bruteforce():
    from oracle import soap
    from synth import config_tiny

    s = config_tiny()
    h = soap.Hypers(**dict(s.hypers, basis="dvr"))
    p = soap.power_spectrum(soap.spherical_expansion(s, h, centres=[0, 17]), h, "full")
    p = p.reshape(2, h.l_max + 1, h.q, h.q)
    for t, i in enumerate([0, 17]):
        ref = soap.power_spectrum_bruteforce(s, h, i)
        assert np.allclose(p[t], ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))
        assert np.max(np.abs(ref)) > 0
