"""Pins of the oracle's brute-force periodic neighbour list."""
import numpy as np

from oracle.neighbours import neighbour_list, neighbours_of_structure
from synth import System, small_cell_system


def _one_atom_cubic(L=1.0):
    return System(np.zeros((1, 3)), np.array([14], np.int32), (np.eye(3) * L)[None], np.ones((1, 3), np.int32),
                  np.array([0, 1], np.int32))


def test_simple_cubic_lattice_counts():
    s = _one_atom_cubic()
    # images at |n| = 1 (6), sqrt 2 (12), sqrt 3 (8), 2 (6)
    assert np.diff(neighbour_list(s, 1.5)["offsets"])[0] == 18
    assert np.diff(neighbour_list(s, 1.8)["offsets"])[0] == 26
    assert np.diff(neighbour_list(s, 2.01)["offsets"])[0] == 32
    # exactly at the cutoff is excluded (strict inequality): r = 1 is representable exactly
    assert np.diff(neighbour_list(s, 1.0)["offsets"])[0] == 0


def test_fcc_nearest_neighbours():
    a = 3.6
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    s = System(basis, np.full(4, 29, np.int32), (np.eye(3) * a)[None], np.ones((1, 3), np.int32), np.array([0, 4], np.int32))
    nl = neighbour_list(s, a / np.sqrt(2) + 0.01)
    assert np.all(np.diff(nl["offsets"]) == 12)


def test_pair_symmetry_and_vectors(tiny_system):
    nl = neighbour_list(tiny_system, 5.0)
    cent = np.repeat(np.arange(tiny_system.n_atoms), np.diff(nl["offsets"]))
    fwd = set(zip(cent.tolist(), nl["nbr_j"].tolist(), map(tuple, nl["shifts"].tolist())))
    bwd = set(zip(nl["nbr_j"].tolist(), cent.tolist(), map(tuple, (-nl["shifts"]).tolist())))
    assert fwd == bwd
    H = tiny_system.cells[0]
    d = tiny_system.positions[nl["nbr_j"]] - tiny_system.positions[cent] + nl["shifts"] @ H
    assert np.allclose(d, nl["rij"], atol=1e-12)
    assert np.all(np.linalg.norm(nl["rij"], axis=1) < 5.0)


def test_matches_scipy_periodic_kdtree(tiny_system):
    # L = 10 = 2 r_cut: each pair is seen through its minimum image only; scipy counts unordered pairs
    from scipy.spatial import cKDTree

    L = tiny_system.cells[0, 0, 0]
    tree = cKDTree(np.mod(tiny_system.positions, L), boxsize=L)
    pairs = tree.query_pairs(5.0)
    nl = neighbour_list(tiny_system, 5.0)
    assert len(nl["nbr_j"]) == 2 * len(pairs)


def test_translation_by_cell_vector_changes_only_shifts():
    s = small_cell_system()
    nl0 = neighbour_list(s, 5.0)
    moved = System(s.positions.copy(), s.species, s.cells, s.pbc, s.struct_offsets, s.hypers)
    moved.positions[2] += s.cells[0, 0] * 2 - s.cells[0, 2]
    nl1 = neighbour_list(moved, 5.0)
    assert np.array_equal(nl0["offsets"], nl1["offsets"])
    assert np.allclose(nl0["rij"][np.argsort(nl0["nbr_j"], kind="stable")].sum(), nl1["rij"][np.argsort(nl1["nbr_j"], kind="stable")].sum())


def test_small_cell_has_self_images_and_sorted_order():
    s = small_cell_system()
    nl = neighbour_list(s, 5.0)
    cent = np.repeat(np.arange(s.n_atoms), np.diff(nl["offsets"]))
    assert np.any(cent == nl["nbr_j"])                      # images of the centre itself
    assert not np.any((cent == nl["nbr_j"]) & np.all(nl["shifts"] == 0, axis=1))
    key = np.stack([cent, nl["nbr_j"], nl["shifts"][:, 0], nl["shifts"][:, 1], nl["shifts"][:, 2]], 1)
    order = np.lexsort(key.T[::-1])
    assert np.array_equal(order, np.arange(len(order)))
    # brute-force counts by explicit enumeration over a generous box of images
    H = s.cells[0]
    for i in range(s.n_atoms):
        cnt = 0
        for j in range(s.n_atoms):
            for n1 in range(-8, 9):
                for n2 in range(-8, 9):
                    for n3 in range(-8, 9):
                        if i == j and n1 == n2 == n3 == 0:
                            continue
                        d = s.positions[j] - s.positions[i] + np.array([n1, n2, n3]) @ H
                        cnt += d @ d < 25.0
        assert cnt == np.diff(nl["offsets"])[i]


def test_non_periodic_axis():
    s = _one_atom_cubic(3.0)
    # in-plane images only: 4 at distance 3, 4 more at 3 sqrt 2 = 4.24
    _, cnt, _, shifts, _ = neighbours_of_structure(s.positions, s.cells[0], [1, 1, 0], 3.5)
    assert cnt[0] == 4 and np.all(shifts[:, 2] == 0)
    _, cnt, _, shifts, _ = neighbours_of_structure(s.positions, s.cells[0], [1, 1, 0], 4.5)
    assert cnt[0] == 8 and np.all(shifts[:, 2] == 0)
