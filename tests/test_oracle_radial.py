"""Pins of the oracle's GTO basis, restricted 1F1, radial integral and spline against independent facts."""
from math import gamma, pi, sqrt

import numpy as np
import pytest

from oracle import gto, hyp1f1, radial

RC, SIG, NMAX, LMAX = 5.0, 0.5, 8, 6


def _quad(f, a, b, n=2000):
    x, w = np.polynomial.legendre.leggauss(200)
    edges = np.linspace(a, b, n // 200 + 1)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        xx = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        tot += np.sum(0.5 * (hi - lo) * w * f(xx))
    return tot


def test_gto_normalisation_and_overlap_by_quadrature():
    # Eq. GTO: N_n makes int x^2 R_n^2 = 1; overlap closed form against direct quadrature
    S = gto.gto_overlap(RC, NMAX)
    for n in range(NMAX):
        for m in range(NMAX):
            q = _quad(lambda x: x * x * gto.gto_radial(x, RC, NMAX)[:, n] * gto.gto_radial(x, RC, NMAX)[:, m], 0.0, 40.0)
            assert abs(q - S[n, m]) < 1e-12
    assert np.allclose(np.diag(S), 1.0, atol=1e-13)


def test_ogto_basis_is_orthonormal():
    T = gto.orthonormalisation(RC, NMAX)
    x = np.linspace(0, 40, 40001)
    R = gto.gto_radial(x, RC, NMAX) @ T.T                      # o-GTO functions
    M = np.array([[_quad(lambda xx: xx * xx * np.interp(xx, x, R[:, a]) * np.interp(xx, x, R[:, b]), 0, 40, 4000)
                   for b in range(NMAX)] for a in range(NMAX)])
    assert np.allclose(M, np.eye(NMAX), atol=1e-6)            # interp-limited accuracy
    S = gto.gto_overlap(RC, NMAX)
    assert np.allclose(T @ S @ T, np.eye(NMAX), atol=1e-9)


def test_inverse_sqrt_accuracy_against_40_digits():
    # S^-1/2 is ill-conditioned (cond S = 5.7e10 at r_cut 6, n_max 16); the FP64 result must be within
    # eps cond(S) of a 40-digit computation of the same closed form
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rc, n = 6.0, 16
    Sm = mpmath.matrix(n, n)
    for i in range(n):
        for j in range(n):
            si = mpmath.mpf(rc) * max(mpmath.sqrt(i), 1) / n
            sj = mpmath.mpf(rc) * max(mpmath.sqrt(j), 1) / n
            di, dj = 1 / (2 * si ** 2), 1 / (2 * sj ** 2)
            Ni = mpmath.sqrt(2 / (si ** (2 * i + 3) * mpmath.gamma(i + mpmath.mpf(3) / 2)))
            Nj = mpmath.sqrt(2 / (sj ** (2 * j + 3) * mpmath.gamma(j + mpmath.mpf(3) / 2)))
            p = mpmath.mpf(i + j + 3) / 2
            Sm[i, j] = Ni * Nj * mpmath.gamma(p) / 2 * (di + dj) ** (-p)
    E, V = mpmath.eigsy(Sm)
    T = np.array((V * mpmath.diag([1 / mpmath.sqrt(e) for e in E]) * V.T).tolist(), dtype=float)
    S = gto.gto_overlap(rc, n)
    assert np.allclose(S, np.array(Sm.tolist(), dtype=float), rtol=1e-14, atol=1e-15)
    err = np.max(np.abs(gto.orthonormalisation(rc, n) - T)) / np.max(np.abs(T))
    assert err < 2.2e-16 * np.linalg.cond(S)


@pytest.mark.parametrize("r", [0.0, 0.3, 1.1, 2.5, 3.7, 4.99])
def test_closed_form_matches_quadrature(r):
    # Eq. rad-int-gto-1 against Eq. radial-integral-gaussian-density by quadrature (scipy Bessel)
    I = radial.raw_integrals(np.array([r]), RC, SIG, NMAX, LMAX)[0]
    for n in range(NMAX):
        for l in range(LMAX + 1):
            q = radial.quadrature_integral(r, n, l, RC, SIG, NMAX)
            assert abs(I[n, l] - q) <= 1e-12 * max(abs(q), 1e-3), (n, l, I[n, l], q)


def test_n_equals_l_closed_form():
    # 1F1(a; a; z) = e^z, so for n = l: I = pi^1.5 N_n c^l r^l (c+d)^-(2l+3)/2 exp(-c d r^2/(c+d))
    c = 1 / (2 * SIG * SIG)
    d = gto.gto_d(RC, NMAX)
    N = gto.gto_norm(RC, NMAX)
    r = np.linspace(0.0, RC, 37)
    I = radial.raw_integrals(r, RC, SIG, NMAX, LMAX)
    for l in range(min(NMAX, LMAX + 1)):
        ref = pi ** 1.5 * N[l] * c ** l * r ** l * (c + d[l]) ** (-(2 * l + 3) / 2) * np.exp(-c * d[l] * r * r / (c + d[l]))
        assert np.allclose(I[:, l, l], ref, rtol=1e-13, atol=1e-300)


def test_kummer_polynomial_case():
    # n - l = 2k >= 0: b - a = -k, Kummer gives 1F1(a;b;z) = e^z 1F1(-k;b;-z), a finite polynomial
    c = 1 / (2 * SIG * SIG)
    d = gto.gto_d(RC, NMAX)
    for n, l in [(2, 0), (4, 2), (6, 0), (7, 3), (5, 1)]:
        a, b = 0.5 * (n + l + 3), l + 1.5
        k = int(round(a - b))
        r = np.linspace(0.05, RC, 23)
        z = c * c * r * r / (c + d[n])
        poly = np.zeros_like(z)
        term = np.ones_like(z)
        for s in range(k + 1):
            poly += term
            term = term * (-k + s) * (-z) / ((b + s) * (s + 1))
        ref = gamma(a) / gamma(b) * np.exp(-c * r * r + z) * poly
        got = hyp1f1.G(a, b, c, d[n], r)
        assert np.allclose(got, ref, rtol=1e-13)


def test_G_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    c = 1 / (2 * 0.4 * 0.4)
    for n in [0, 3, 7, 11, 15]:
        for l in [0, 1, 4, 9, 12]:
            d = float(gto.gto_d(6.0, 16)[n])
            a, b = 0.5 * (n + l + 3), l + 1.5
            for r in [0.0, 0.4, 1.7, 3.3, 5.2, 6.0]:
                z = c * c * r * r / (c + d)
                ref = mpmath.gamma(a) / mpmath.gamma(b) * mpmath.exp(-c * r * r) * mpmath.hyp1f1(a, b, z)
                got = hyp1f1.G(a, b, c, d, np.array([r]))[0]
                assert abs(got - float(ref)) <= 2e-13 * abs(float(ref)), (n, l, r, got, float(ref))


def test_downward_recurrences_hold():
    # the two relations of Eq. 1f1-recurrence, on the oracle's direct evaluations
    c = 2.0
    d = gto.gto_d(RC, NMAX)[3]
    r = np.linspace(0.1, 5.9, 30)
    z = c * c * r * r / (c + d)
    for n, l in [(0, 0), (3, 2), (7, 6), (5, 9)]:
        a, b = 0.5 * (n + l + 3), l + 1.5
        lhs1 = hyp1f1.G(a + 1, b + 1, c, d, r)
        rhs1 = hyp1f1.recurrence_step_a1b1(hyp1f1.G(a + 2, b + 3, c, d, r), hyp1f1.G(a + 1, b + 2, c, d, r), b, z)
        assert np.allclose(lhs1, rhs1, rtol=1e-12)
        lhs2 = hyp1f1.G(a, b, c, d, r)
        rhs2 = hyp1f1.recurrence_step_ab(hyp1f1.G(a + 1, b + 2, c, d, r), hyp1f1.G(a + 1, b + 1, c, d, r), a, b, z)
        assert np.allclose(lhs2, rhs2, rtol=1e-12)


def test_series_and_asymptotic_agree_beyond_switch():
    for a, b in [(3.0, 4.5), (6.0, 1.5), (10.5, 13.5), (9.0, 1.5)]:
        zs = hyp1f1.switch_point(a, b)
        assert np.isfinite(zs)
        z = np.array([zs * 1.01, zs * 1.5, zs * 3])
        ser = hyp1f1.series_scaled(a, b, z, -z)
        asy, _ = hyp1f1.asymptotic_scaled(a, b, z, -z)
        assert np.allclose(ser, asy, rtol=2e-13)


def test_zero_distance_only_l0():
    I = radial.integrals(np.array([0.0]), RC, SIG, NMAX, LMAX)[0]
    assert np.all(I[:, 1:] == 0.0)
    assert np.all(np.abs(I[:, 0]) > 0)


def test_derivative_vs_central_difference():
    r = np.array([0.35, 1.5, 2.9, 4.4, 4.97])
    _, dI = radial.integrals(r, RC, SIG, NMAX, LMAX, derivative=True)
    h = 1e-5
    fd = (radial.integrals(r + h, RC, SIG, NMAX, LMAX) - radial.integrals(r - h, RC, SIG, NMAX, LMAX)) / (2 * h)
    assert np.allclose(dI, fd, atol=2e-8, rtol=1e-6)
    # at r = 0 a one-sided difference
    _, d0 = radial.integrals(np.array([0.0]), RC, SIG, NMAX, LMAX, derivative=True)
    fwd = (radial.integrals(np.array([h]), RC, SIG, NMAX, LMAX) - radial.integrals(np.array([0.0]), RC, SIG, NMAX, LMAX)) / h
    assert np.allclose(d0[0], fwd[0], atol=1e-4)
    assert np.all(d0[0][:, 0] == 0.0) and np.all(d0[0][:, 2:] == 0.0)   # only l = 1 has a slope at r = 0


def test_spline_reproduces_cubic_exactly_and_matches_scipy():
    from scipy.interpolate import CubicSpline

    delta = 0.25
    x = np.arange(21) * delta
    f = lambda t: 0.3 - 1.2 * t + 0.7 * t ** 2 - 0.05 * t ** 3
    df = lambda t: -1.2 + 1.4 * t - 0.15 * t ** 2
    y2 = radial.spline_second_derivatives(f(x), df(0.0), df(x[-1]), delta)
    t = np.linspace(0, x[-1], 333)
    val, dval = radial.spline_eval(t, f(x), y2, delta, derivative=True)
    assert np.allclose(val, f(t), atol=1e-12)
    assert np.allclose(dval, df(t), atol=1e-11)
    g = np.sin(1.3 * x) * np.exp(-0.2 * x)
    dg0 = 1.3
    dgM = 1.3 * np.cos(1.3 * x[-1]) * np.exp(-0.2 * x[-1]) - 0.2 * g[-1]
    y2 = radial.spline_second_derivatives(g, dg0, dgM, delta)
    ref = CubicSpline(x, g, bc_type=((1, dg0), (1, dgM)))
    assert np.allclose(radial.spline_eval(t, g, y2, delta), ref(t), atol=1e-13)


def test_spline_accuracy_and_fourth_order_convergence():
    s128 = radial.RadialSpline(RC, SIG, NMAX, LMAX, n_intervals=128)
    s256 = radial.RadialSpline(RC, SIG, NMAX, LMAX, n_intervals=256)
    e128, e256 = s128.midpoint_error(), s256.midpoint_error()
    assert 10.0 < e128 / e256 < 22.0                           # O(h^4): ratio ~ 16
    auto = radial.RadialSpline(RC, SIG, NMAX, LMAX, accuracy=1e-8)
    assert auto.midpoint_error() <= 1e-8
