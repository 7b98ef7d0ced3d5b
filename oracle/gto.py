"""GTO radial basis of Eq. GTO (Sec. 'GTO radial basis') and its Löwdin orthogonalisation.

R_n(r) = N_n r^n exp(-d_n r^2),  d_n = 1/(2 sigma_n^2),  sigma_n = r_cut max(sqrt(n), 1) / n_max,
N_n^2 = 2 / (sigma_n^(2n+3) Gamma(n + 3/2)),  0 <= n < n_max.

The o-GTO basis is |n; o-GTO> = sum_n' [S^-1/2]_nn' |n'; GTO>, with S the overlap matrix of the GTOs.
"""
from __future__ import annotations

from math import gamma, sqrt

import numpy as np


def gto_sigma(r_cut: float, n_max: int) -> np.ndarray:
    n = np.arange(n_max, dtype=np.float64)
    return r_cut * np.maximum(np.sqrt(n), 1.0) / n_max


def gto_d(r_cut: float, n_max: int) -> np.ndarray:
    s = gto_sigma(r_cut, n_max)
    return 1.0 / (2.0 * s * s)


def gto_norm(r_cut: float, n_max: int) -> np.ndarray:
    s = gto_sigma(r_cut, n_max)
    return np.array([sqrt(2.0 / (s[n] ** (2 * n + 3) * gamma(n + 1.5))) for n in range(n_max)])


def gto_radial(x: np.ndarray, r_cut: float, n_max: int) -> np.ndarray:
    """R_n(x) for all n: shape [len(x), n_max]."""
    x = np.asarray(x, dtype=np.float64)[:, None]
    n = np.arange(n_max)[None, :]
    return gto_norm(r_cut, n_max)[None, :] * x ** n * np.exp(-gto_d(r_cut, n_max)[None, :] * x * x)


def gto_overlap(r_cut: float, n_max: int) -> np.ndarray:
    """S_nn' = int_0^inf x^2 R_n(x) R_n'(x) dx = N_n N_n' Gamma((n+n'+3)/2) / (2 (d_n + d_n')^((n+n'+3)/2))."""
    N = gto_norm(r_cut, n_max)
    d = gto_d(r_cut, n_max)
    S = np.empty((n_max, n_max))
    for n in range(n_max):
        for m in range(n_max):
            p = 0.5 * (n + m + 3)
            S[n, m] = N[n] * N[m] * 0.5 * gamma(p) * (d[n] + d[m]) ** (-p)
    return S


def inverse_sqrt(S: np.ndarray) -> np.ndarray:
    """Symmetric inverse square root from an FP64 eigendecomposition."""
    w, V = np.linalg.eigh(S)
    if np.min(w) <= 0:
        raise ValueError("overlap matrix is not positive definite")
    return (V * (1.0 / np.sqrt(w))[None, :]) @ V.T


def orthonormalisation(r_cut: float, n_max: int) -> np.ndarray:
    """[S^-1/2]_nn' of the GTO overlap matrix."""
    return inverse_sqrt(gto_overlap(r_cut, n_max))
