"""Pins of the oracle's real spherical harmonics: closed forms, scipy, addition theorem, orthonormality, gradient."""
from math import pi, sqrt

import numpy as np

from oracle import ylm


def _dirs(n, seed=0):
    v = np.random.default_rng(seed).standard_normal((n, 3))
    v[0] = [0.0, 0.0, 2.0]          # north pole
    v[1] = [0.0, 0.0, -0.7]         # south pole
    v[2] = [1.5, 0.0, 0.0]
    return v


def test_closed_forms_up_to_l2():
    v = _dirs(40)
    u = v / np.linalg.norm(v, axis=1)[:, None]
    x, y, z = u.T
    Y = ylm.real_ylm(v, 2)
    c1 = sqrt(3 / (4 * pi))
    ref = {
        (0, 0): np.full_like(x, 1 / (2 * sqrt(pi))),
        (1, -1): c1 * y, (1, 0): c1 * z, (1, 1): c1 * x,
        (2, -2): 0.5 * sqrt(15 / pi) * x * y, (2, -1): 0.5 * sqrt(15 / pi) * y * z,
        (2, 0): 0.25 * sqrt(5 / pi) * (3 * z * z - 1), (2, 1): 0.5 * sqrt(15 / pi) * x * z,
        (2, 2): 0.25 * sqrt(15 / pi) * (x * x - y * y),
    }
    for (l, m), r in ref.items():
        assert np.allclose(Y[:, ylm.lm_index(l, m)], r, atol=1e-14)


def test_matches_scipy_up_to_stated_phase():
    from scipy.special import sph_harm_y

    v = _dirs(30)
    u = v / np.linalg.norm(v, axis=1)[:, None]
    th, ph = np.arccos(np.clip(u[:, 2], -1, 1)), np.arctan2(u[:, 1], u[:, 0])
    L = 12
    Y = ylm.real_ylm(v, L)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            cy = sph_harm_y(l, abs(m), th, ph)          # complex, with Condon-Shortley phase
            ref = cy.real if m == 0 else sqrt(2) * (-1) ** m * (cy.real if m > 0 else cy.imag)
            assert np.allclose(Y[:, ylm.lm_index(l, m)], ref, atol=1e-12), (l, m)


def test_addition_theorem():
    from numpy.polynomial import legendre

    a, b = _dirs(25, 1), _dirs(25, 2)
    ua, ub = a / np.linalg.norm(a, axis=1)[:, None], b / np.linalg.norm(b, axis=1)[:, None]
    L = 14
    Ya, Yb = ylm.real_ylm(a, L), ylm.real_ylm(b, L)
    cos = np.sum(ua * ub, axis=1)
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = np.sum(Ya[:, sl] * Yb[:, sl], axis=1)
        coeff = np.zeros(l + 1)
        coeff[l] = 1
        rhs = (2 * l + 1) / (4 * pi) * legendre.legval(cos, coeff)
        assert np.allclose(lhs, rhs, atol=1e-12)


def test_orthonormality_by_quadrature():
    L = 8
    xg, wg = np.polynomial.legendre.leggauss(L + 2)
    nphi = 2 * L + 3
    phi = 2 * pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    v = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * pi / nphi)[None, :]).reshape(-1)
    Y = ylm.real_ylm(v, L)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye((L + 1) ** 2), atol=1e-12)


def test_gradient_vs_central_difference_and_tangency():
    v = _dirs(20, 3) * 2.3
    L = 10
    _, dY = ylm.real_ylm(v, L, gradient=True)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (ylm.real_ylm(v + e, L) - ylm.real_ylm(v - e, L)) / (2 * h)
        assert np.allclose(dY[:, :, k], fd, atol=1e-7)
    # Y depends on direction only: the gradient is orthogonal to r
    assert np.allclose(np.einsum("pkx,px->pk", dY, v), 0.0, atol=1e-12)
