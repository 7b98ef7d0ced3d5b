"""Real spherical harmonics Y_lm(r^) and their gradients with respect to the vector r (Sec. 'Spherical Harmonics').

Reading (the paper names the Limpanuparb-Milthorpe recurrences but fixes no convention): orthonormal real
harmonics without the Condon-Shortley phase, stored at index lm = l^2 + l + m,
  m > 0: sqrt(2) N_lm P_l^m(cos t) cos(m phi)
  m = 0: N_l0 P_l(cos t)
  m < 0: sqrt(2) N_l|m| P_l^|m|(cos t) sin(|m| phi)
with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).

On the unit sphere sin^m(t) e^{i m phi} = (x + i y)^m, so with P_l^m(z) = (1 - z^2)^{m/2} Pt_l^m(z),
Y_lm = sqrt(2) N_lm Pt_l^m(z) Re[(x + i y)^m] (and Im for m < 0): a polynomial in the unit-vector components.
Pt obeys the usual associated-Legendre three-term recurrence in l. The gradient in r is the gradient of that
polynomial in u = r/|r| projected on the tangent plane and divided by |r|.
"""
from __future__ import annotations

from math import factorial, pi, sqrt

import numpy as np


def lm_index(l: int, m: int) -> int:
    return l * l + l + m


def _norm(l: int, m: int) -> float:
    return sqrt((2 * l + 1) / (4 * pi) * factorial(l - m) / factorial(l + m))


def _legendre_tilde(z: np.ndarray, l_max: int):
    """Pt_l^m(z) and dPt_l^m/dz for 0 <= m <= l <= l_max: arrays [l_max+1, l_max+1, len(z)] indexed [l, m]."""
    P = np.zeros((l_max + 1, l_max + 1, z.size))
    dP = np.zeros_like(P)
    for m in range(l_max + 1):
        dfact = 1.0
        for k in range(1, 2 * m, 2):
            dfact *= k  # (2m - 1)!!
        P[m, m] = dfact
        if m + 1 <= l_max:
            P[m + 1, m] = (2 * m + 1) * z * P[m, m]
            dP[m + 1, m] = (2 * m + 1) * P[m, m]
        for l in range(m + 2, l_max + 1):
            P[l, m] = ((2 * l - 1) * z * P[l - 1, m] - (l + m - 1) * P[l - 2, m]) / (l - m)
            dP[l, m] = ((2 * l - 1) * (P[l - 1, m] + z * dP[l - 1, m]) - (l + m - 1) * dP[l - 2, m]) / (l - m)
    return P, dP


def real_ylm(vec: np.ndarray, l_max: int, gradient: bool = False):
    """Y_lm(vec/|vec|) for vectors [P, 3]: [P, (l_max+1)^2]; with gradient=True also dY/dvec [P, (l_max+1)^2, 3]."""
    vec = np.atleast_2d(np.asarray(vec, dtype=np.float64))
    r = np.sqrt(np.sum(vec * vec, axis=1))
    u = vec / r[:, None]
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    P, dP = _legendre_tilde(z, l_max)
    w = (x + 1j * y)
    powers = np.ones((l_max + 1, vec.shape[0]), dtype=np.complex128)
    for m in range(1, l_max + 1):
        powers[m] = powers[m - 1] * w
    C = powers.real
    S = powers.imag
    nlm = (l_max + 1) ** 2
    Y = np.zeros((vec.shape[0], nlm))
    dYu = np.zeros((vec.shape[0], nlm, 3))
    for l in range(l_max + 1):
        for m in range(0, l + 1):
            Nlm = _norm(l, m)
            if m == 0:
                Y[:, lm_index(l, 0)] = Nlm * P[l, 0]
                dYu[:, lm_index(l, 0), 2] = Nlm * dP[l, 0]
                continue
            f = sqrt(2.0) * Nlm
            Cm1, Sm1 = C[m - 1], S[m - 1]
            # cosine harmonic
            Y[:, lm_index(l, m)] = f * P[l, m] * C[m]
            dYu[:, lm_index(l, m), 0] = f * P[l, m] * m * Cm1
            dYu[:, lm_index(l, m), 1] = f * P[l, m] * (-m) * Sm1
            dYu[:, lm_index(l, m), 2] = f * dP[l, m] * C[m]
            # sine harmonic
            Y[:, lm_index(l, -m)] = f * P[l, m] * S[m]
            dYu[:, lm_index(l, -m), 0] = f * P[l, m] * m * Sm1
            dYu[:, lm_index(l, -m), 1] = f * P[l, m] * m * Cm1
            dYu[:, lm_index(l, -m), 2] = f * dP[l, m] * S[m]
    if not gradient:
        return Y
    # project on the tangent plane: dY/dvec = (I - u u^T) dY/du / r
    radial = np.einsum("pkj,pj->pk", dYu, u)
    dY = (dYu - radial[:, :, None] * u[:, None, :]) / r[:, None, None]
    return Y, dY
