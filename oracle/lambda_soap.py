"""nu = 2 equivariant features (lambda-SOAP) from the density coefficients, in FP64: test infrastructure, like all of
oracle/.

Sec. "Experimental features" builds equivariants from the same coefficients by the symmetrised correlation of
Eq. body-order-x at nu = 2 without the final contraction to an invariant:
    T^{lambda mu}_{(a1 n1 l1)(a2 n2 l2)} = sum_{m1 m2} <l1 m1; l2 m2 | lambda mu> c_{a1 n1 l1 m1} c_{a2 n2 l2 m2}
with Clebsch-Gordan coefficients <..|..> (complex, Condon-Shortley convention). Readings:
* the average over improper rotations (k = 0, 1 in Eq. body-order-x) keeps the proper tensors, l1 + l2 + lambda
  even; pseudotensors are not computed;
* the coefficients are those of the real harmonics of oracle/ylm (no Condon-Shortley phase). The coupling is carried
  into that basis with the unitary U, Y^R = U Y^CS, of each l: R[m1', m2', mu] = sum U_lambda[mu, M] <..|lambda M>
  conj(U_l1[m1', m1]) conj(U_l2[m2', m2]); for l1 + l2 + lambda even R is real;
* T for (l2, l1) is the transpose of T for (l1, l2) (the CG symmetry with l1 + l2 + lambda even), so only pairs with
  l1 <= l2 are formed, ordered by l1 then l2, each as [2 lambda + 1][Q][Q] with q = a n_max + n;
* lambda = 0 reproduces (-1)^l times the power spectrum of Eq. nu2-basis-coupled with its (2l+1)^-1/2 factor.
"""
from __future__ import annotations

from math import factorial, sqrt

import numpy as np


def clebsch_gordan(l1: int, m1: int, l2: int, m2: int, L: int, M: int) -> float:
    """<l1 m1; l2 m2 | L M> for integer angular momenta, by Racah's closed form in exact integer arithmetic."""
    l1, m1, l2, m2, L, M = (int(v) for v in (l1, m1, l2, m2, L, M))
    if m1 + m2 != M or not (abs(l1 - l2) <= L <= l1 + l2) or abs(m1) > l1 or abs(m2) > l2 or abs(M) > L:
        return 0.0
    pref_num = (2 * L + 1) * factorial(L + l1 - l2) * factorial(L - l1 + l2) * factorial(l1 + l2 - L)
    pref_num *= factorial(L + M) * factorial(L - M) * factorial(l1 - m1) * factorial(l1 + m1)
    pref_num *= factorial(l2 - m2) * factorial(l2 + m2)
    pref_den = factorial(l1 + l2 + L + 1)
    s = 0.0
    for k in range(0, l1 + l2 + 1):
        a = [k, l1 + l2 - L - k, l1 - m1 - k, l2 + m2 - k, L - l2 + m1 + k, L - l1 - m2 + k]
        if min(a) < 0:
            continue
        den = 1
        for v in a:
            den *= factorial(v)
        s += (-1) ** k / den
    return sqrt(pref_num / pref_den) * s


def real_from_condon_shortley(l: int) -> np.ndarray:
    """U [2l+1][2l+1] (rows: real m' = -l..l, columns: complex m = -l..l) with Y^R_{lm'} = sum_m U[m', m] Y^CS_{lm}.

    With Z^m = N P^|m| e^{i m phi} (no phase), Y^CS_m = (-1)^m Z^m for m > 0 and Z^m for m <= 0, while the real
    harmonics are Z^0, (Z^m + Z^-m)/sqrt 2 (m > 0) and (Z^m - Z^-m)/(i sqrt 2) (index -m)."""
    U = np.zeros((2 * l + 1, 2 * l + 1), dtype=complex)
    U[l, l] = 1.0
    for m in range(1, l + 1):
        U[l + m, l + m] = (-1) ** m / sqrt(2)
        U[l + m, l - m] = 1 / sqrt(2)
        U[l - m, l + m] = (-1) ** m / (1j * sqrt(2))
        U[l - m, l - m] = -1 / (1j * sqrt(2))
    return U


def real_coupling(l1: int, l2: int, L: int) -> np.ndarray:
    """R [2l1+1][2l2+1][2L+1] coupling real-basis coefficients of l1 and l2 to real-basis rank L (l1 + l2 + L even)."""
    C = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * L + 1))
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            M = m1 + m2
            if abs(M) <= L:
                C[m1 + l1, m2 + l2, M + L] = clebsch_gordan(l1, m1, l2, m2, L, M)
    U1, U2, UL = real_from_condon_shortley(l1), real_from_condon_shortley(l2), real_from_condon_shortley(L)
    R = np.einsum("uM,abM,xa,yb->xyu", UL, C, np.conj(U1), np.conj(U2))
    if np.max(np.abs(R.imag)) > 1e-12:
        raise ValueError(f"coupling ({l1}, {l2}) -> {L} is not real in this basis")
    return R.real


def pairs(l_max: int, lam: int):
    """(l1, l2) with l1 <= l2 <= l_max, |l1 - l2| <= lambda <= l1 + l2 and l1 + l2 + lambda even, by l1 then l2."""
    return [(l1, l2) for l1 in range(l_max + 1) for l2 in range(l1, l_max + 1)
            if abs(l1 - l2) <= lam <= l1 + l2 and (l1 + l2 + lam) % 2 == 0]


def equivariants(c, hypers, lam: int) -> np.ndarray:
    """T [n_centres][n_pairs][2 lambda + 1][Q][Q] from c [n_centres][S][n_max][(l_max+1)^2]."""
    h = hypers
    n_c = c.shape[0]
    C = np.asarray(c, dtype=np.float64).reshape(n_c, h.q, h.n_lm)
    P = pairs(h.l_max, lam)
    out = np.zeros((n_c, len(P), 2 * lam + 1, h.q, h.q))
    for k, (l1, l2) in enumerate(P):
        R = real_coupling(l1, l2, lam)
        A = C[:, :, l1 * l1:(l1 + 1) ** 2]
        B = C[:, :, l2 * l2:(l2 + 1) ** 2]
        out[:, k] = np.einsum("xyu,iax,iby->iuab", R, A, B)
    return out
