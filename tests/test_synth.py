"""The seeded synthetic workloads follow their stated recipes (cell, atom count, density, minimum distance, species
mix, expansion parameters) and are reproducible from their seeds. These generators stand in for the paper's
datasets; both the oracle and the GPU path take their inputs from them, so a drifted recipe would change every
workload at once without failing any parity test.
"""
from math import pi

import numpy as np
import pytest

from synth import config_batch, config_diff, config_large, config_mlp, config_tiny

spatial = pytest.importorskip("scipy.spatial")


def _cubic_side(s, k=0):
    cell = s.cells[k]
    assert np.allclose(cell, np.eye(3) * cell[0, 0]) and np.all(s.pbc[k] == 1)
    return float(cell[0, 0])


def _min_distance_and_mean_neighbours(pos, L, r_cut):
    tree = spatial.cKDTree(np.mod(pos, L), boxsize=L)
    d, _ = tree.query(np.mod(pos, L), k=2)
    n_pairs = len(tree.query_pairs(r_cut))
    return float(np.min(d[:, 1])), 2.0 * n_pairs / len(pos)


def _hypers(s, r_cut, sigma, n_max, l_max, species):
    h = s.hypers
    assert (h["r_cut"], h["sigma"], h["n_max"], h["l_max"], h["smooth_width"]) == (r_cut, sigma, n_max, l_max, 0.5)
    assert sorted(h["species"]) == sorted(species) and set(np.unique(s.species)) <= set(species)


def test_tiny():
    s = config_tiny()
    _hypers(s, 5.0, 0.5, 8, 6, [14])
    L = _cubic_side(s)
    assert s.n_atoms == 64 and s.n_structures == 1 and L == 10.0 and np.all(s.species == 14)
    dmin, _ = _min_distance_and_mean_neighbours(s.positions, L, 5.0)
    assert dmin >= 2.0


def test_batch():
    s = config_batch()
    _hypers(s, 5.0, 0.5, 12, 9, [1, 6, 7, 8])
    counts = np.diff(s.struct_offsets)
    assert s.n_structures == 512 and counts.min() >= 64 and counts.max() <= 216 and counts.sum() == s.n_atoms
    # atom counts uniform on 64..216: mean 140, and both ends of the range are reached in 512 draws
    assert abs(counts.mean() - 140.0) < 4 * 44.2 / np.sqrt(512) and counts.min() < 70 and counts.max() > 210
    # four species drawn uniformly
    frac = np.array([np.mean(s.species == z) for z in (1, 6, 7, 8)])
    assert np.all(np.abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / s.n_atoms))
    dmins, nbrs = [], []
    for k in range(s.n_structures):
        a, b = s.struct_offsets[k], s.struct_offsets[k + 1]
        L = _cubic_side(s, k)
        assert abs((b - a) / L ** 3 - 0.05) < 1e-12
        dmin, nb = _min_distance_and_mean_neighbours(s.positions[a:b], L, 5.0)
        dmins.append(dmin)
        nbrs.append(nb * (b - a))
    assert min(dmins) >= 1.8
    # about 4/3 pi r_cut^3 rho = 26 neighbours per centre (the hard core removes a few)
    assert 22.0 < sum(nbrs) / s.n_atoms < 27.0


def test_diff():
    s = config_diff()
    _hypers(s, 5.5, 0.4, 8, 6, [1, 6])
    L = _cubic_side(s)
    assert s.n_atoms == 4096 and abs(4096 / L ** 3 - 0.05) < 1e-12
    assert np.sum(s.species == 1) == 2048 and np.sum(s.species == 6) == 2048
    dmin, nb = _min_distance_and_mean_neighbours(s.positions, L, 5.5)
    assert dmin >= 1.8 and 30.0 < nb < 4 / 3 * pi * 5.5 ** 3 * 0.05 + 1.0


def test_large():
    s = config_large()
    _hypers(s, 6.0, 0.5, 10, 8, [1, 6, 8])
    L = _cubic_side(s)
    assert s.n_atoms == 32768 and abs(32768 / L ** 3 - 0.1) < 1e-12
    assert [int(np.sum(s.species == z)) for z in (1, 6, 8)] == [16384, 8192, 8192]
    dmin, nb = _min_distance_and_mean_neighbours(s.positions, L, 6.0)
    # the neighbour-count regime of the large workload: about 90 neighbours per atom
    assert dmin >= 1.0 and 87.0 < nb < 4 / 3 * pi * 6.0 ** 3 * 0.1 + 1.0


def test_mlp():
    s = config_mlp()
    _hypers(s, 6.0, 0.5, 16, 12, [1, 5, 6, 7, 8, 9, 15, 16])
    L = _cubic_side(s)
    assert s.n_atoms == 8192 and abs(8192 / L ** 3 - 0.06) < 1e-12
    counts = np.array([np.sum(s.species == z) for z in (1, 5, 6, 7, 8, 9, 15, 16)])
    assert np.all(np.abs(counts - 1024) < 5 * np.sqrt(8192 * (1 / 8) * (7 / 8)))
    dmin, _ = _min_distance_and_mean_neighbours(s.positions, L, 6.0)
    assert dmin >= 1.6


def test_seeds_reproduce_and_differ():
    a, b, c = config_batch(seed=2, n_structures=4), config_batch(seed=2, n_structures=4), config_batch(seed=3, n_structures=4)
    assert np.array_equal(a.positions, b.positions) and np.array_equal(a.species, b.species)
    assert np.array_equal(a.struct_offsets, b.struct_offsets)
    assert not (a.positions.shape == c.positions.shape and np.array_equal(a.positions, c.positions))
    # the full batch workload's first cells are the same cells as the 4-cell case of the same seed
    full = config_batch(seed=2)
    assert np.array_equal(full.positions[: a.n_atoms], a.positions)
