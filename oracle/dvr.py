"""DVR radial basis (Sec. 'DVR radial basis', Eq. rad-int-dvr) in FP64: test infrastructure, like all of oracle/.

The basis functions vanish at every Gauss-Legendre point on [0, r_cut + 3 sigma] but one; the paper writes
<x|n> = sqrt(w_n) delta(x - x_n), read with the radial measure as int x^2 R_n(x) f(x) dx = x_n sqrt(w_n) f(x_n), which
gives the printed prefactor x_n sqrt(w_n). Projecting the Gaussian density
exp(-a |x - r|^2), a = 1/(2 sigma^2), of one neighbour at distance r on R_n(x) Y_lm(x^) uses
    int dOmega_x Y_lm(x^) exp(-a |x - r|^2) = 4 pi exp(-a (x^2 + r^2)) i_l(2 a x r) Y_lm(r^),
with i_l the modified spherical Bessel function of the first kind, so that
    I^DVR_nl(r) = 4 pi x_n sqrt(w_n) exp(-a (x_n^2 + r^2)) i_l(2 a x_n r).
Reading: the printed Eq. rad-int-dvr leaves out the constant 4 pi and the factor exp(-a r^2) of the density; both are
kept here (the latter makes the integral decay with r, as the GTO form does). The basis is orthonormal by construction,
so no S^-1/2 step follows. The products exp(-a(x - r)^2) e^{-z} i_l(z) are evaluated with the exponentially scaled
Bessel function so that nothing overflows.
"""
from __future__ import annotations

from math import pi

import numpy as np
from scipy import special


def nodes(r_cut: float, sigma: float, n_max: int):
    """Gauss-Legendre points x_n and weights w_n on [0, r_cut + 3 sigma]."""
    t, w = np.polynomial.legendre.leggauss(n_max)
    half = 0.5 * (r_cut + 3.0 * sigma)
    return half * (t + 1.0), half * w


def scaled_bessel_i(l_max: int, z):
    """e^-z i_l(z) for l = 0..l_max at z >= 0: array [len(z), l_max + 1]."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    out = np.zeros((z.size, l_max + 1))
    small = z < 1e-4
    zs = z[~small]
    for l in range(l_max + 1):
        out[~small, l] = np.sqrt(np.pi / (2.0 * zs)) * special.ive(l + 0.5, zs)
        # series i_l(z) = z^l / (2l+1)!! (1 + z^2 / (2 (2l+3)) + z^4 / (8 (2l+3)(2l+5)))
        zz = z[small]
        dfact = np.prod(np.arange(1, 2 * l + 2, 2, dtype=np.float64))
        out[small, l] = np.exp(-zz) * zz ** l / dfact * (1.0 + zz * zz / (2.0 * (2 * l + 3))
                                                          + zz ** 4 / (8.0 * (2 * l + 3) * (2 * l + 5)))
    return out


def integrals(r, r_cut: float, sigma: float, n_max: int, l_max: int, derivative: bool = False):
    """I^DVR_nl(r) (and dI/dr): arrays [len(r), n_max, l_max + 1]."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    a = 1.0 / (2.0 * sigma * sigma)
    x, w = nodes(r_cut, sigma, n_max)
    out = np.zeros((r.size, n_max, l_max + 1))
    dout = np.zeros((r.size, n_max, l_max + 1))
    for n in range(n_max):
        z = 2.0 * a * x[n] * r
        e = scaled_bessel_i(l_max + 1, z)                         # e^-z i_l(z), l = 0..l_max+1
        g = 4.0 * pi * x[n] * np.sqrt(w[n]) * np.exp(-a * (x[n] - r) ** 2)
        out[:, n, :] = g[:, None] * e[:, :l_max + 1]
        if derivative:
            # d/dz [e^-z i_l] = e^-z (i_{l+1} + (l/z) i_l - i_l); the l/z term tends to 1/3 (l = 1) or 0 at z = 0
            lz = np.zeros((r.size, l_max + 1))
            nz = z > 0
            for l in range(1, l_max + 1):
                lz[nz, l] = l / z[nz] * e[nz, l]
                if l == 1:
                    lz[~nz, l] = 1.0 / 3.0
            de = e[:, 1:l_max + 2] + lz - e[:, :l_max + 1]
            dout[:, n, :] = g[:, None] * (2.0 * a * (x[n] - r)[:, None] * e[:, :l_max + 1] + 2.0 * a * x[n] * de)
    if derivative:
        return out, dout
    return out
