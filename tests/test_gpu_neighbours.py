"""GPU neighbour list against the brute-force FP64 oracle: bit-exact indices and shifts, FP32-accurate vectors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.neighbours import neighbour_list  # noqa: E402
from synth import System, config_batch, config_tiny, random_cell_atoms, small_cell_system  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _gpu_pairs(rg, system, hypers=None):
    h = dict(system.hypers if hypers is None else hypers)
    calc = rg.SoapCalculator(**h)
    ds = rg.DeviceSystem.from_numpy(system)
    pl = calc.neighbours(ds)
    return calc, ds, {k: getattr(pl, k).cpu().numpy() for k in ("offsets", "nbr_j", "shifts", "rij")}


def _assert_same(gpu, ref, centres=None):
    if centres is None:
        assert np.array_equal(gpu["offsets"], ref["offsets"])
        assert np.array_equal(gpu["nbr_j"], ref["nbr_j"])
        assert np.array_equal(gpu["shifts"], ref["shifts"])
        rij = gpu["rij"]
    else:
        segs = [np.arange(gpu["offsets"][c], gpu["offsets"][c + 1]) for c in centres]
        idx = np.concatenate(segs) if segs else np.zeros(0, np.int64)
        assert np.array_equal(np.array([len(s) for s in segs]), np.diff(ref["offsets"]))
        assert np.array_equal(gpu["nbr_j"][idx], ref["nbr_j"])
        assert np.array_equal(gpu["shifts"][idx], ref["shifts"])
        rij = gpu["rij"][idx]
    d = ref["rij"]
    assert np.allclose(rij[:, :3], d, rtol=0, atol=2e-7 * np.maximum(1.0, np.abs(d)).max())
    assert np.allclose(rij[:, 3], np.linalg.norm(d, axis=1), rtol=3e-7)


def test_tiny_bitexact(rg):
    s = config_tiny()
    _, _, gpu = _gpu_pairs(rg, s)
    _assert_same(gpu, neighbour_list(s, s.hypers["r_cut"]))


def test_small_triclinic_cell_with_self_images_unwrapped_positions(rg):
    for seed in (11, 12, 13):
        s = small_cell_system(seed=seed, n_atoms=7, L=4.0)
        _, _, gpu = _gpu_pairs(rg, s)
        ref = neighbour_list(s, s.hypers["r_cut"])
        _assert_same(gpu, ref)
        cent = np.repeat(np.arange(s.n_atoms), np.diff(ref["offsets"]))
        assert np.any(cent == ref["nbr_j"])


def test_pairs_at_the_cutoff_follow_the_fp64_definition(rg):
    # pairs placed within a few ulp of r_cut, in cubic and skewed cells, one pair per structure
    rc = 5.0
    pos, cells, offs = [], [], [0]
    for k in range(-6, 7):
        for cell in (np.eye(3) * 11.0, np.array([[11.0, 0, 0], [3.0, 11.5, 0], [1.0, -2.0, 12.0]])):
            a = np.array([1.0, 2.0, 3.0])
            u = np.array([0.6, 0.0, 0.8])
            b = a + u * (rc + k * 1e-15)
            pos += [a, b]
            cells.append(cell)
            offs.append(offs[-1] + 2)
    # an exactly representable distance of r_cut: excluded
    pos += [np.array([0.5, 0.5, 0.5]), np.array([5.5, 0.5, 0.5])]
    cells.append(np.eye(3) * 20.0)
    offs.append(offs[-1] + 2)
    s = System(np.array(pos), np.full(len(pos), 14, np.int32), np.stack(cells), np.ones((len(cells), 3), np.int32),
               np.array(offs, np.int32), dict(r_cut=rc, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=[14]))
    _, _, gpu = _gpu_pairs(rg, s)
    ref = neighbour_list(s, rc)
    _assert_same(gpu, ref)
    assert len(ref["nbr_j"]) > 0


def test_empty_structures_and_isolated_atoms(rg):
    pos = np.array([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0], [9.0, 9.0, 9.0]])
    cells = np.stack([np.eye(3) * 30.0, np.eye(3) * 30.0, np.eye(3) * 30.0])
    s = System(pos, np.array([14, 14, 14], np.int32), cells, np.array([[1, 1, 1], [0, 0, 0], [1, 1, 1]], np.int32),
               np.array([0, 1, 1, 3], np.int32), dict(r_cut=5.0, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=[14]))
    _, _, gpu = _gpu_pairs(rg, s)
    assert np.array_equal(gpu["offsets"], [0, 0, 0, 0])


def test_non_periodic_axis(rg):
    base = small_cell_system(seed=3, n_atoms=6, L=6.0)
    s = System(base.positions, base.species, base.cells, np.array([[1, 0, 1]], np.int32), base.struct_offsets, base.hypers)
    _, _, gpu = _gpu_pairs(rg, s)
    _assert_same(gpu, neighbour_list(s, s.hypers["r_cut"]))


def test_batch_full_size_sampled_and_symmetric(rg):
    s = config_batch()
    _, _, gpu = _gpu_pairs(rg, s)
    rng = np.random.default_rng(0)
    centres = np.sort(rng.choice(s.n_atoms, 24, replace=False))
    centres = np.concatenate([[0, s.n_atoms - 1], centres])
    _assert_same(gpu, neighbour_list(s, s.hypers["r_cut"], centres), centres)
    # the relation is symmetric: (i, j, n) present iff (j, i, -n) present
    cent = np.repeat(np.arange(s.n_atoms), np.diff(gpu["offsets"]))
    fwd = np.stack([cent, gpu["nbr_j"], *gpu["shifts"].T], 1)
    bwd = np.stack([gpu["nbr_j"], cent, *(-gpu["shifts"]).T], 1)
    fwd = fwd[np.lexsort(fwd.T[::-1])]
    bwd = bwd[np.lexsort(bwd.T[::-1])]
    assert np.array_equal(fwd, bwd)


def test_capacity_and_unknown_species_errors(rg):
    import ctypes as C

    import torch

    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    sys_c = ds.c_struct()
    off = torch.empty(s.n_atoms + 1, dtype=torch.int64, device="cuda")
    P = C.c_int64(0)
    lib = rg._lib.lib()
    st = lib.rascal_neighbours(calc._ctx, C.byref(sys_c), 10, C.c_void_p(off.data_ptr()), None, None, None, C.byref(P))
    assert st == rg._lib.RASCAL_E_CAPACITY and P.value > 10
    bad = rg.DeviceSystem.from_numpy(System(s.positions, np.full(s.n_atoms, 6, np.int32), s.cells, s.pbc,
                                            s.struct_offsets, s.hypers))
    with pytest.raises(rg.RascalError) as e:
        calc.neighbours(bad)
    assert e.value.code == rg._lib.RASCAL_E_ARG
    # the context stays usable after an error
    pl = calc.neighbours(ds)
    assert pl.n_pairs == P.value


def test_centres_with_more_than_128_neighbours(rg):
    # 532 atoms in a 16 A cell with r_cut 7: 164..202 neighbours per centre, more than a warp sorts in shared
    # memory, so every segment goes through the global overflow sort
    L, n = 16.0, 532
    rng = np.random.Generator(np.random.PCG64(51))
    pos = random_cell_atoms(n, np.eye(3) * L, 1.2, rng)
    s = System(pos, np.full(n, 6, np.int32), (np.eye(3) * L)[None], np.ones((1, 3), np.int32), np.array([0, n], np.int32),
               dict(r_cut=7.0, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=[6]))
    _, _, gpu = _gpu_pairs(rg, s)
    ref = neighbour_list(s, 7.0)
    assert np.diff(ref["offsets"]).min() > 128
    _assert_same(gpu, ref)


def _expect_status(rg, system, code, text):
    calc = rg.SoapCalculator(**system.hypers)
    with pytest.raises(rg.RascalError) as e:
        calc.neighbours(rg.DeviceSystem.from_numpy(system))
    assert e.value.code == code, (e.value.code, str(e.value))
    assert text in str(e.value)
    # the context keeps working after the error
    t = config_tiny()
    calc2 = rg.SoapCalculator(**t.hypers)
    assert calc2.neighbours(rg.DeviceSystem.from_numpy(t)).n_pairs > 0


HYP = dict(r_cut=5.0, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=[14])


def _one_cell(pos, cell):
    pos = np.asarray(pos, np.float64)
    return System(pos, np.full(len(pos), 14, np.int32), np.asarray(cell, np.float64)[None], np.ones((1, 3), np.int32),
                  np.array([0, len(pos)], np.int32), dict(HYP))


def test_coincident_atoms_are_a_geometry_error(rg):
    pos = [[1.0, 2.0, 3.0], [4.0, 4.0, 4.0], [1.0, 2.0, 3.0]]
    _expect_status(rg, _one_cell(pos, np.eye(3) * 12.0), rg._lib.RASCAL_E_GEOMETRY, "coincident")
    # an atom on top of another atom's periodic image is coincident too
    pos = [[1.0, 2.0, 3.0], [13.0, 2.0, 3.0]]
    _expect_status(rg, _one_cell(pos, np.eye(3) * 12.0), rg._lib.RASCAL_E_GEOMETRY, "coincident")


def test_singular_and_too_thin_cells_are_refused(rg):
    singular = np.array([[10.0, 0.0, 0.0], [0.0, 10.0, 0.0], [5.0, 5.0, 0.0]])
    _expect_status(rg, _one_cell([[1.0, 1.0, 1.0], [3.0, 2.0, 1.0]], singular), rg._lib.RASCAL_E_GEOMETRY, "singular")
    thin = np.diag([10.0, 10.0, 0.05])  # perpendicular width 0.05 < r_cut / 64
    _expect_status(rg, _one_cell([[1.0, 1.0, 0.01], [3.0, 2.0, 0.02]], thin), rg._lib.RASCAL_E_UNSUPPORTED, "thinner")


def test_non_finite_positions_are_refused(rg):
    for bad in (np.nan, np.inf, -np.inf):
        pos = [[1.0, 2.0, 3.0], [4.0, bad, 4.0], [6.0, 6.0, 6.0]]
        _expect_status(rg, _one_cell(pos, np.eye(3) * 12.0), rg._lib.RASCAL_E_ARG, "not finite")
