"""Pins of the oracle's nu = 2 equivariants (lambda-SOAP): the Clebsch-Gordan coefficients against a library
routine and their orthogonality, the coupling of two real harmonics to one (a closed form that fixes every phase
convention), the lambda = 0 reduction to the power spectrum, and rotation covariance of the features."""
import numpy as np
import pytest

from oracle import lambda_soap as ls
from oracle import soap, ylm


def test_clebsch_gordan_against_sympy_and_orthogonality():
    wigner = pytest.importorskip("sympy.physics.wigner")
    rng = np.random.default_rng(3)
    for _ in range(40):
        l1, l2 = rng.integers(0, 5, size=2)
        L = rng.integers(abs(l1 - l2), l1 + l2 + 1)
        m1 = rng.integers(-l1, l1 + 1)
        m2 = rng.integers(-l2, l2 + 1)
        ref = float(wigner.clebsch_gordan(int(l1), int(l2), int(L), int(m1), int(m2), int(m1 + m2)))
        assert np.isclose(ls.clebsch_gordan(l1, m1, l2, m2, L, m1 + m2), ref, rtol=1e-13, atol=1e-15)
    l1, l2 = 3, 2
    for L in range(1, 6):
        for Lp in range(1, 6):
            for M in (-1, 0, 1):
                s = sum(ls.clebsch_gordan(l1, m1, l2, M - m1, L, M) * ls.clebsch_gordan(l1, m1, l2, M - m1, Lp, M)
                        for m1 in range(-l1, l1 + 1) if abs(M - m1) <= l2)
                assert np.isclose(s, 1.0 if L == Lp else 0.0, atol=1e-13)


def test_coupling_of_two_real_harmonics_is_one_real_harmonic():
    """sum R[m1, m2, mu] Y_l1m1(u) Y_l2m2(u) = sqrt((2l1+1)(2l2+1)/(4 pi (2L+1))) <l1 0; l2 0|L 0> Y_Lmu(u)."""
    rng = np.random.default_rng(5)
    u = rng.normal(size=(7, 3))
    Y = ylm.real_ylm(u, 8)
    for l1 in range(5):
        for l2 in range(l1, 5):
            for L in range(abs(l1 - l2), l1 + l2 + 1):
                if (l1 + l2 + L) % 2:
                    continue
                R = ls.real_coupling(l1, l2, L)
                lhs = np.einsum("xyu,px,py->pu", R, Y[:, l1 * l1:(l1 + 1) ** 2], Y[:, l2 * l2:(l2 + 1) ** 2])
                k = np.sqrt((2 * l1 + 1) * (2 * l2 + 1) / (4 * np.pi * (2 * L + 1))) * ls.clebsch_gordan(l1, 0, l2, 0, L, 0)
                assert np.allclose(lhs, k * Y[:, L * L:(L + 1) ** 2], atol=1e-12)


def test_lambda_zero_is_the_power_spectrum_up_to_sign():
    from synth import config_tiny

    s = config_tiny()
    h = soap.Hypers(**s.hypers)
    c = soap.spherical_expansion(s, h, centres=[0, 11, 30])
    T = ls.equivariants(c, h, 0)
    assert [p for p in ls.pairs(h.l_max, 0)] == [(l, l) for l in range(h.l_max + 1)]
    p = soap.power_spectrum(c, h, "full").reshape(3, h.l_max + 1, h.q, h.q)
    for l in range(h.l_max + 1):
        assert np.allclose(T[:, l, 0], (-1) ** l * p[:, l], rtol=1e-12, atol=1e-14 * np.max(np.abs(p[:, l])))


def _real_wigner(R, L):
    """Real Wigner matrix D with Y_L(R u) = D Y_L(u), fitted on many directions (exact for a rotation)."""
    rng = np.random.default_rng(9)
    u = rng.normal(size=(64, 3))
    Yu = ylm.real_ylm(u, L)[:, L * L:(L + 1) ** 2]
    YRu = ylm.real_ylm(u @ R.T, L)[:, L * L:(L + 1) ** 2]
    D, *_ = np.linalg.lstsq(Yu, YRu, rcond=None)
    return D.T


@pytest.mark.parametrize("lam", [1, 2, 3])
def test_rotation_covariance(lam):
    from synth import small_cell_system

    s = small_cell_system(seed=17, n_atoms=7, L=4.8, hypers=dict(r_cut=4.0, sigma=0.5, n_max=3, l_max=4,
                                                                 smooth_width=0.6, species=[1, 8]))
    h = soap.Hypers(**s.hypers)
    rng = np.random.default_rng(lam)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Rm = q * np.sign(np.linalg.det(q))  # proper rotation
    T0 = ls.equivariants(soap.spherical_expansion(s, h, centres=[0, 4]), h, lam)
    s.positions, s.cells = s.positions @ Rm.T, s.cells @ Rm.T
    T1 = ls.equivariants(soap.spherical_expansion(s, h, centres=[0, 4]), h, lam)
    D = _real_wigner(Rm, lam)
    assert np.max(np.abs(T0)) > 0
    assert np.allclose(T1, np.einsum("uv,ikvab->ikuab", D, T0), atol=1e-10 * np.max(np.abs(T0)))
    # inversion: with l1 + l2 + lambda even the features change like Y_lambda, by (-1)^lambda (polar tensors)
    s.positions, s.cells = -s.positions, -s.cells
    T2 = ls.equivariants(soap.spherical_expansion(s, h, centres=[0, 4]), h, lam)
    assert np.allclose(T2, (-1) ** lam * T1, atol=1e-10 * np.max(np.abs(T0)))


def test_swapped_pair_is_the_transpose():
    """T for (l2, l1), formed directly with the coupling in that order, equals the transpose of T for (l1, l2)."""
    from synth import config_tiny

    s = config_tiny()
    h = soap.Hypers(**s.hypers)
    c = soap.spherical_expansion(s, h, centres=[2]).reshape(1, h.q, h.n_lm)
    for l1, l2, L in [(1, 3, 2), (2, 3, 1), (0, 2, 2)]:
        A, B = c[:, :, l1 * l1:(l1 + 1) ** 2], c[:, :, l2 * l2:(l2 + 1) ** 2]
        T12 = np.einsum("xyu,iax,iby->iuab", ls.real_coupling(l1, l2, L), A, B)
        T21 = np.einsum("xyu,iax,iby->iuab", ls.real_coupling(l2, l1, L), B, A)
        assert np.allclose(T21, np.swapaxes(T12, 2, 3), atol=1e-13 * np.max(np.abs(T12)))
