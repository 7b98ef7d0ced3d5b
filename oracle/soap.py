"""Density coefficients, power spectrum, additive linear energy and its gradients, in FP64.

c^i_{a n l m} = sum_{j in A_i, a_j = a} f_cut(r_ji) I^o_nl(r_ji) Y_lm(r^_ji)      (Eq. spherical_expansion_coefficients_gaussians)
p^i_{(a1 n1)(a2 n2) l} = (2l+1)^-1/2 sum_m c^i_{a1 n1 l m} c^i_{a2 n2 l m}         (Eq. nu2-basis-coupled, real basis)
E = sum_i w_{a_i} . p^i                                                           (Eq. additive-energy-model, linear E(A_i))
dE/dr_k = sum_i sum_j dE_i/dr_ji (delta_jk - delta_ik)                             (Eq. energy-derivative)
dE/deta = sum_i sum_j dE_i/dr_ji (x) r_ji                                         (Eq. energy-virial)

Readings:
* f_cut is the cosine cutoff: 1 for r <= r_cut - w, (1 + cos(pi (r - r_cut + w)/w))/2 up to r_cut, 0 beyond;
* the centre does not contribute to its own density unless include_center is set (then the r = 0 term,
  where only l = 0 survives, is added to the centre's own species block);
* for a real density the printed sum_m (-1)^m c_lm c_l(-m) equals sum_m c_lm c_lm in the real basis;
* the (2l+1)^-1/2 factor is kept (flag ps_norm);
* species are ordered by their sorted labels; the combined index is q = a n_max + n;
* FULL layout stores p[i][l][q1][q2]; PACKED stores q1 <= q2 row-major, p[i][l][k];
* the linear model has one Gaussian weight vector per centre species over the PACKED features;
* the virial is written as V[alpha][beta] = sum g_alpha r_beta with g = dE/dr_ji.
"""
from __future__ import annotations

from math import pi, sqrt

import numpy as np

from . import dvr, radial, ylm
from .neighbours import neighbour_list


class Hypers:
    def __init__(self, r_cut, sigma, n_max, l_max, species, smooth_width=0.5, orthonormal=True, include_center=False,
                 ps_norm=True, basis="gto", **_ignored):
        self.r_cut = float(r_cut)
        self.sigma = float(sigma)
        self.n_max = int(n_max)
        self.l_max = int(l_max)
        self.species = sorted(int(s) for s in species)
        self.smooth_width = float(smooth_width)
        self.orthonormal = bool(orthonormal)
        self.include_center = bool(include_center)
        self.ps_norm = bool(ps_norm)
        self.basis = str(basis)  # "gto" (Eq. rad-int-gto-1, o-GTO unless orthonormal is off) or "dvr" (Eq. rad-int-dvr)

    @property
    def n_species(self):
        return len(self.species)

    @property
    def n_lm(self):
        return (self.l_max + 1) ** 2

    @property
    def q(self):
        return self.n_species * self.n_max

    def n_features(self, layout="packed"):
        Q = self.q
        per_l = Q * (Q + 1) // 2 if layout == "packed" else Q * Q
        return (self.l_max + 1) * per_l

    def species_index(self, labels):
        lut = {s: a for a, s in enumerate(self.species)}
        return np.array([lut[int(x)] for x in labels], dtype=np.int64)


def cutoff(r, r_cut, width, derivative=False):
    r = np.asarray(r, dtype=np.float64)
    t = (r - r_cut + width) / width
    f = np.where(r <= r_cut - width, 1.0, np.where(r >= r_cut, 0.0, 0.5 * (1.0 + np.cos(pi * t))))
    if not derivative:
        return f
    df = np.where((r > r_cut - width) & (r < r_cut), -0.5 * pi / width * np.sin(pi * t), 0.0)
    return f, df


def _radial(r, h: Hypers, derivative=False, radial_fn=None):
    if radial_fn is not None:
        return radial_fn(r, derivative)
    if h.basis == "dvr":
        return dvr.integrals(r, h.r_cut, h.sigma, h.n_max, h.l_max, derivative)
    return radial.integrals(r, h.r_cut, h.sigma, h.n_max, h.l_max, h.orthonormal, derivative)


def spherical_expansion(system, hypers: Hypers, centres=None, nl=None, radial_fn=None):
    """c for the listed centres (default all): [n_c, n_species, n_max, (l_max+1)^2] FP64.

    radial_fn(r, derivative) may replace the exact integral (e.g. the FP64 spline mode)."""
    h = hypers
    if nl is None:
        nl = neighbour_list(system, h.r_cut, centres)
    centres = nl["centres"]
    a_all = h.species_index(system.species)
    rij = nl["rij"]
    out = np.zeros((centres.size, h.n_species, h.n_max, h.n_lm))
    if rij.shape[0]:
        r = np.sqrt(np.sum(rij * rij, axis=1))
        fc = cutoff(r, h.r_cut, h.smooth_width)
        I = _radial(r, h, radial_fn=radial_fn)                     # [P, n, l]
        Y = ylm.real_ylm(rij, h.l_max)                             # [P, lm]
        lidx = np.array([l for l in range(h.l_max + 1) for _ in range(2 * l + 1)])
        contrib = fc[:, None, None] * I[:, :, lidx] * Y[:, None, :]  # [P, n, lm]
        pair_centre = np.repeat(np.arange(centres.size), np.diff(nl["offsets"]))
        pair_species = a_all[nl["nbr_j"]]
        np.add.at(out, (pair_centre, pair_species), contrib)
    if h.include_center:
        I0 = _radial(np.zeros(1), h, radial_fn=radial_fn)[0]       # [n, l]
        f0 = cutoff(0.0, h.r_cut, h.smooth_width)
        y00 = 1.0 / (2.0 * sqrt(pi))
        for t, i in enumerate(centres):
            out[t, a_all[i], :, 0] += f0 * I0[:, 0] * y00
    return out


def _packed_pairs(Q):
    return [(q1, q2) for q1 in range(Q) for q2 in range(q1, Q)]


def power_spectrum(c, hypers: Hypers, layout="packed"):
    """p from c: FULL [n_c, l_max+1, Q, Q] or PACKED [n_c, l_max+1, Q(Q+1)/2]."""
    h = hypers
    n_c = c.shape[0]
    Q = h.q
    C = c.reshape(n_c, Q, h.n_lm)
    full = np.zeros((n_c, h.l_max + 1, Q, Q))
    for l in range(h.l_max + 1):
        Cl = C[:, :, l * l: (l + 1) * (l + 1)]                      # [n_c, Q, 2l+1]
        k = 1.0 / sqrt(2 * l + 1) if h.ps_norm else 1.0
        full[:, l] = k * np.einsum("iam,ibm->iab", Cl, Cl)
    if layout == "full":
        return full
    iu = np.triu_indices(Q)
    return full[:, :, iu[0], iu[1]]


def power_spectrum_bruteforce(system, hypers: Hypers, centre: int, radial_fn=None):
    """Y_lm-free power spectrum of one centre through the addition theorem (a pin for power_spectrum):

    p_{(a1 n1)(a2 n2) l} = k_l (2l+1)/(4 pi) sum_{j: a_j=a1} sum_{k: a_k=a2} f_j f_k I_{n1 l}(r_j) I_{n2 l}(r_k) P_l(r^_j . r^_k)
    with k_l = (2l+1)^-1/2, returned in the FULL layout [l_max+1, Q, Q]."""
    from numpy.polynomial import legendre

    h = hypers
    nl = neighbour_list(system, h.r_cut, [centre])
    rij = nl["rij"]
    a = h.species_index(system.species)[nl["nbr_j"]]
    r = np.sqrt(np.sum(rij * rij, axis=1))
    f = cutoff(r, h.r_cut, h.smooth_width)
    I = _radial(r, h, radial_fn=radial_fn)
    u = rij / r[:, None]
    cosg = np.clip(u @ u.T, -1.0, 1.0)
    Q = h.q
    out = np.zeros((h.l_max + 1, Q, Q))
    for l in range(h.l_max + 1):
        coeffs = np.zeros(l + 1)
        coeffs[l] = 1.0
        Pl = legendre.legval(cosg, coeffs)
        k = (1.0 / sqrt(2 * l + 1) if h.ps_norm else 1.0) * (2 * l + 1) / (4 * pi)
        A = np.zeros((Q, r.size))
        for n in range(h.n_max):
            A[a * h.n_max + n, np.arange(r.size)] = f * I[:, n, l]
        out[l] = k * A @ Pl @ A.T
    return out


def linear_energy(p_packed, centre_species, weights):
    """E = sum_i w[a_i] . p_i over PACKED features; returns (E, per-centre energies)."""
    p = p_packed.reshape(p_packed.shape[0], -1)
    e = np.einsum("if,if->i", weights[centre_species], p)
    return float(np.sum(e)), e


def adjoint_coefficients(c, hypers: Hypers, grad_p_packed):
    """dE/dc for E = sum_i grad_p_i . p_i (PACKED layout): chat_l = k_l (W_l + W_l^T) C_l per centre.

    W_l holds the packed gradient on and above the diagonal and zeros below it."""
    h = hypers
    n_c = c.shape[0]
    Q = h.q
    C = c.reshape(n_c, Q, h.n_lm)
    G = grad_p_packed.reshape(n_c, h.l_max + 1, Q * (Q + 1) // 2)
    iu = np.triu_indices(Q)
    chat = np.zeros_like(C)
    for l in range(h.l_max + 1):
        W = np.zeros((n_c, Q, Q))
        W[:, iu[0], iu[1]] = G[:, l]
        k = 1.0 / sqrt(2 * l + 1) if h.ps_norm else 1.0
        sl = slice(l * l, (l + 1) * (l + 1))
        chat[:, :, sl] = k * np.einsum("iab,ibm->iam", W + np.transpose(W, (0, 2, 1)), C[:, :, sl])
    return chat.reshape(c.shape)


def energy_gradients(system, hypers: Hypers, weights, radial_fn=None, centres=None, grad_p=None, nl=None):
    """Forces F = -dE/dr [N,3] and virial V = sum_pairs dE/dr_ji (x) r_ji [n_structures,3,3] for the linear model.

    dE_i/dr_ji = sum_{n l m} chat^i_{a_j n l m} grad_r [f(r) I_nl(r) Y_lm(r^)], evaluated exactly per pair.
    centres: optional subset of centre atoms; the result is then the gradient of sum_{i in centres} E_i only.
    grad_p: optional dE/dp per centre [n_centres, F] (PACKED) in place of the linear model's weights[a_i], for any
    energy that depends on the atoms through the power spectrum only (Eq. gpr-force-order).
    nl: optional neighbour list of those centres from neighbour_list (saves recomputing it)."""
    h = hypers
    if nl is None:
        nl = neighbour_list(system, h.r_cut, centres)
    cidx = nl["centres"]
    c = spherical_expansion(system, h, nl=nl, radial_fn=radial_fn)
    a_all = h.species_index(system.species)
    p = power_spectrum(c, h, "packed")
    grad_p = (weights[a_all[cidx]] if grad_p is None else np.asarray(grad_p, dtype=np.float64)).reshape(p.shape)
    chat = adjoint_coefficients(c, h, grad_p)                       # [N, S, n, lm]
    rij = nl["rij"]
    forces = np.zeros((system.n_atoms, 3))
    virial = np.zeros((system.n_structures, 3, 3))
    if rij.shape[0] == 0:
        return forces, virial
    r = np.sqrt(np.sum(rij * rij, axis=1))
    u = rij / r[:, None]
    f, df = cutoff(r, h.r_cut, h.smooth_width, derivative=True)
    I, dI = _radial(r, h, derivative=True, radial_fn=radial_fn)
    Y, dY = ylm.real_ylm(rij, h.l_max, gradient=True)
    lidx = np.array([l for l in range(h.l_max + 1) for _ in range(2 * l + 1)])
    centre_row = np.repeat(np.arange(cidx.size), np.diff(nl["offsets"]))
    centre = cidx[centre_row]
    j = nl["nbr_j"]
    ch = chat[centre_row, a_all[j]]                                 # [P, n, lm]
    R = f[:, None, None] * I[:, :, lidx]                           # radial part f I, [P, n, lm]
    dR = (df[:, None, None] * I[:, :, lidx] + f[:, None, None] * dI[:, :, lidx])
    # grad [R Y] = dR/dr u Y + R grad Y
    s1 = np.einsum("pnk,pnk,pk->p", ch, dR, Y)
    g = s1[:, None] * u + np.einsum("pnk,pnk,pkx->px", ch, R, dY)   # dE/dr_ji per pair
    # a pair whose j is an image of the centre moves with it: its two terms cancel (Appendix B), so it is skipped
    other = j != centre
    np.add.at(forces, j[other], -g[other])
    np.add.at(forces, centre[other], g[other])
    sid = system.structure_of_atom()[centre]
    np.add.at(virial, sid, np.einsum("pa,pb->pab", g, rij))
    return forces, virial


def total_energy(system, hypers: Hypers, weights, radial_fn=None):
    c = spherical_expansion(system, hypers, radial_fn=radial_fn)
    p = power_spectrum(c, hypers, "packed")
    return linear_energy(p, hypers.species_index(system.species), weights)[0]
