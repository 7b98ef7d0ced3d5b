"""Sparse Gaussian-process energy model with the polynomial kernel, in FP64: test infrastructure, like all of oracle/.

E(A_i) = sum_{I in M, a_I = a_i} x_I k_zeta(M_I, A_i)                 (Eq. sparse-gp, one model per centre species)
k_zeta(M_I, A_i) = (sum_q M_Iq p_iq)^zeta                             (polynomial kernel, Sec. "Sparse kernel models")
dk_zeta/dp_iq = zeta M_Iq k_(zeta-1)(M_I, A_i)
dE/dp_i = sum_I x_I dk_zeta/dp_i, summed over the active set first    (Eq. gpr-force-order)

Reading: the kernel acts on unit-normalised feature vectors when `normalize` is set (the usual form of the SOAP
polynomial kernel; the paper's equations leave the normalisation to the representation): p^_i = p_i / |p_i| and
M^_I = M_I / |M_I|. Then dE/dp_i = (G_i - (G_i . p^_i) p^_i) / |p_i| with G_i = sum_I x_I zeta k_(zeta-1) M^_I, and
G_i . p^_i = zeta E_i, since every term of G_i . p^_i is zeta x_I k_zeta. With `normalize` off the vectors are used
as given. The features are the PACKED power spectrum (or any selected subset of it), one row per centre.
"""
from __future__ import annotations

import numpy as np


def _unit(v):
    n = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
    return v / np.where(n > 0, n, 1.0), n[..., 0]


def kernel(p, sparse, zeta: int, normalize: bool = True):
    """k_zeta between every row of p [N, F] and every sparse point [n, F]: [N, n]."""
    p = np.asarray(p, dtype=np.float64)
    sparse = np.asarray(sparse, dtype=np.float64)
    if normalize:
        p, _ = _unit(p)
        sparse, _ = _unit(sparse)
    return (p @ sparse.T) ** zeta


def energies(p, centre_species, sparse, sparse_species, weights, zeta: int, normalize: bool = True):
    """Per-centre energies E_i [N]: each centre sees only the sparse points of its own species."""
    p = np.asarray(p, dtype=np.float64)
    E = np.zeros(p.shape[0])
    for s in np.unique(centre_species):
        rows = np.flatnonzero(centre_species == s)
        cols = np.flatnonzero(sparse_species == s)
        if cols.size == 0:
            continue
        E[rows] = kernel(p[rows], sparse[cols], zeta, normalize) @ np.asarray(weights, dtype=np.float64)[cols]
    return E


def grad_p(p, centre_species, sparse, sparse_species, weights, zeta: int, normalize: bool = True):
    """dE_i/dp_i [N, F], the derivative of the kernel summed over the active set before anything else."""
    p = np.asarray(p, dtype=np.float64)
    sparse = np.asarray(sparse, dtype=np.float64)
    x = np.asarray(weights, dtype=np.float64)
    out = np.zeros_like(p)
    for s in np.unique(centre_species):
        rows = np.flatnonzero(centre_species == s)
        cols = np.flatnonzero(sparse_species == s)
        if cols.size == 0:
            continue
        P, M = p[rows], sparse[cols]
        if normalize:
            P, norm = _unit(P)
            M, _ = _unit(M)
        K1 = (P @ M.T) ** (zeta - 1)                                  # k_(zeta-1)
        G = (zeta * K1 * x[cols][None, :]) @ M                        # sum_I x_I dk/dp^
        if normalize:
            E = ((P @ M.T) ** zeta) @ x[cols]
            G = (G - zeta * E[:, None] * P) / np.where(norm > 0, norm, 1.0)[:, None]
        out[rows] = G
    return out
