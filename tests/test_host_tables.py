"""Tables the library builds on the host, through its C ABI on the CPU (no GPU): the Gauss-Legendre points and
weights of the DVR radial basis (Eq. rad-int-dvr) against numpy's leggauss and the exactness of the rule, and the
real-basis coupling tables of the nu = 2 equivariants (Eq. body-order-x) against the FP64 oracle.
"""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_08814_gb300 import _lib, build

    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    return _lib.lib()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 16, 33, 64])
def test_gauss_legendre_points_and_weights(lib, n):
    X = 6.5
    x, w = np.zeros(n), np.zeros(n)
    assert lib.rascal_debug_gauss_legendre(n, X, _ptr(x), _ptr(w)) == 0
    t, wt = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(x) > 0)
    assert np.max(np.abs(x - 0.5 * X * (t + 1.0))) <= 4e-15 * X
    assert np.max(np.abs(w - 0.5 * X * wt)) <= 1e-13 * X / n
    # the n-point rule integrates polynomials of degree 2n - 1 on [0, X] exactly
    for k in (0, 1, 2 * n - 1):
        assert abs(np.sum(w * x ** k) - X ** (k + 1) / (k + 1)) <= 1e-12 * X ** (k + 1) / (k + 1)


def test_gauss_legendre_rejects_bad_arguments(lib):
    x, w = np.zeros(4), np.zeros(4)
    assert lib.rascal_debug_gauss_legendre(0, 1.0, _ptr(x), _ptr(w)) == -1
    assert lib.rascal_debug_gauss_legendre(65, 1.0, _ptr(x), _ptr(w)) == -1
    assert lib.rascal_debug_gauss_legendre(4, 0.0, _ptr(x), _ptr(w)) == -1


def test_real_coupling_tables_match_the_oracle(lib):
    from oracle import lambda_soap as ols

    worst = 0.0
    for l1 in range(5):
        for l2 in range(5):
            for lam in range(abs(l1 - l2), l1 + l2 + 1):
                if (l1 + l2 + lam) % 2:
                    continue
                R = np.zeros((2 * lam + 1, 2 * l1 + 1, 2 * l2 + 1), np.float32)
                assert lib.rascal_debug_real_coupling(l1, l2, lam, _ptr(R)) == 0
                ref = np.transpose(ols.real_coupling(l1, l2, lam), (2, 0, 1))  # [m1][m2][mu] -> [mu][m1][m2]
                worst = max(worst, float(np.max(np.abs(R.astype(np.float64) - ref))))
    # one FP32 rounding of entries of magnitude <= 1
    assert worst <= 6e-8, worst


def test_real_coupling_rejects_odd_and_non_triangular_ranks(lib):
    R = np.zeros(1000, np.float32)
    assert lib.rascal_debug_real_coupling(1, 1, 1, _ptr(R)) == -1   # l1 + l2 + lambda odd
    assert lib.rascal_debug_real_coupling(1, 1, 4, _ptr(R)) == -1   # outside |l1 - l2| .. l1 + l2
    assert lib.rascal_debug_real_coupling(16, 0, 16, _ptr(R)) == -1  # above the largest l
