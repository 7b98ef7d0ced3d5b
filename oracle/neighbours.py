"""Brute-force periodic neighbour list: every (i, j, n) with |r_j - r_i + n H| < r_cut (Appendix B).

Appendix B defines the environment A_i by the vectors r_ji = r_j - r_i with r_ji < r_cut, where j runs over the
periodic images as well. The shift n = (n1, n2, n3) counts cell vectors: the image of j sits at
r_j + n1 h1 + n2 h2 + n3 h3. The pair (j = i, n = 0) is the centre itself and is left out; other images of i
are kept.

Readings:
* positions are used as given, without wrapping into the cell, so the shifts refer to the input positions;
* the displacement is evaluated left to right in FP64 with every operation rounded on its own,
  d = (r_j - r_i) + ((n1 h1 + n2 h2) + n3 h3), and the pair is kept when ((dx dx + dy dy) + dz dz) < r_cut r_cut
  (strict, as "r_ji < r_cut");
* along a non-periodic axis only n_k = 0 is used;
* the output is sorted by (i, j, n1, n2, n3).
"""
from __future__ import annotations

import numpy as np


def _perp_widths(cell: np.ndarray) -> np.ndarray:
    vol = abs(np.linalg.det(cell))
    return np.array([vol / np.linalg.norm(np.cross(cell[(k + 1) % 3], cell[(k + 2) % 3])) for k in range(3)])


def neighbours_of_structure(positions: np.ndarray, cell: np.ndarray, pbc, r_cut: float, centres=None):
    """Neighbour list of one structure.

    Returns (centres, counts, nbr_j, shifts, rij): for each listed centre its neighbour count, then the
    concatenated neighbour indices (local to the structure), integer shifts [P,3] and FP64 vectors r_ji [P,3].
    """
    positions = np.asarray(positions, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    n_atoms = positions.shape[0]
    if centres is None:
        centres = np.arange(n_atoms)
    frac = positions @ np.linalg.inv(cell)
    spread = frac.max(axis=0) - frac.min(axis=0) if n_atoms else np.zeros(3)
    widths = _perp_widths(cell)
    K = [int(np.ceil(r_cut / widths[k] + spread[k])) + 1 if pbc[k] else 0 for k in range(3)]
    grid = np.array(np.meshgrid(np.arange(-K[0], K[0] + 1), np.arange(-K[1], K[1] + 1),
                                np.arange(-K[2], K[2] + 1), indexing="ij")).reshape(3, -1).T
    # shift vectors, evaluated left to right: (n1 h1 + n2 h2) + n3 h3
    sv = (grid[:, 0:1].astype(np.float64) * cell[0][None, :] + grid[:, 1:2].astype(np.float64) * cell[1][None, :]) \
        + grid[:, 2:3].astype(np.float64) * cell[2][None, :]
    rc2 = r_cut * r_cut
    counts, js, ns, ds = [], [], [], []
    for i in centres:
        rel = positions - positions[i][None, :]                    # r_j - r_i
        d = rel[:, None, :] + sv[None, :, :]                       # [N, n_shift, 3]
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        mask = d2 < rc2
        jj, kk = np.nonzero(mask)
        shifts = grid[kk]
        keep = ~((jj == i) & np.all(shifts == 0, axis=1))
        jj, shifts, dd = jj[keep], shifts[keep], d[jj[keep], kk[keep]]
        order = np.lexsort((shifts[:, 2], shifts[:, 1], shifts[:, 0], jj))
        counts.append(len(order))
        js.append(jj[order])
        ns.append(shifts[order])
        ds.append(dd[order])
    if not counts:
        return np.asarray(centres), np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros((0, 3), np.int32), np.zeros((0, 3))
    return (np.asarray(centres), np.asarray(counts, dtype=np.int64), np.concatenate(js).astype(np.int32),
            np.concatenate(ns).astype(np.int32), np.concatenate(ds))


def neighbour_list(system, r_cut: float, centres=None):
    """Neighbour list of a batch System in its flat (global) atom numbering.

    centres: optional global atom indices to restrict to (sampled parity checks); default all atoms.
    Returns dict(offsets [n_c+1] int64, nbr_j [P] int32 global, shifts [P,3] int32, rij [P,3] float64,
    centres [n_c] int64).
    """
    off = system.struct_offsets
    sid = system.structure_of_atom()
    if centres is None:
        centres = np.arange(system.n_atoms)
    centres = np.asarray(centres, dtype=np.int64)
    counts = np.zeros(centres.size, dtype=np.int64)
    js, ns, ds = [], [], []
    # group by structure, keep the caller's centre order
    results = {}
    for s in np.unique(sid[centres]) if centres.size else []:
        local = centres[sid[centres] == s] - off[s]
        a, b = off[s], off[s + 1]
        cs, cnt, jj, nn, dd = neighbours_of_structure(system.positions[a:b], system.cells[s], system.pbc[s], r_cut, local)
        starts = np.concatenate([[0], np.cumsum(cnt)])
        for t, c in enumerate(cs):
            results[int(c + a)] = (jj[starts[t]:starts[t + 1]] + a, nn[starts[t]:starts[t + 1]], dd[starts[t]:starts[t + 1]])
    for t, c in enumerate(centres):
        jj, nn, dd = results[int(c)]
        counts[t] = jj.size
        js.append(jj)
        ns.append(nn)
        ds.append(dd)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    if js:
        return dict(offsets=offsets, nbr_j=np.concatenate(js).astype(np.int32), shifts=np.concatenate(ns).astype(np.int32),
                    rij=np.concatenate(ds), centres=centres)
    return dict(offsets=offsets, nbr_j=np.zeros(0, np.int32), shifts=np.zeros((0, 3), np.int32), rij=np.zeros((0, 3)),
                centres=centres)
