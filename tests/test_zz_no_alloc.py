"""The neighbour search entry point that allocates no device memory (rascal_neighbours_noalloc).

Callers such as an MD engine whose device memory is held by its own pool allocator, or a time-stepping loop that
must not hit cudaMalloc/cudaFree (both synchronise the device), cannot let the library grow a scratch arena. This
entry point takes its scratch from a fixed device array compiled into the library. The test calls it through the
C ABI twice in a row, on two different systems, and checks each result against rascal_neighbours on the same
input: offsets, neighbour indices and shifts bit-exact, r_ji vectors identical (same kernels, same arithmetic).
The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from synth import System, config_batch, config_tiny, random_cell_atoms, small_cell_system  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _noalloc(rg, calc, ds, capacity):
    import torch

    lib = rg._lib.lib()
    N = ds.n_atoms
    off = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    nbr = torch.empty(capacity, dtype=torch.int32, device="cuda")
    sh = torch.empty((capacity, 3), dtype=torch.int32, device="cuda")
    rij = torch.empty((capacity, 4), dtype=torch.float32, device="cuda")
    P = C.c_int64(0)
    calc._bind_stream()
    sys_c = ds.c_struct()
    st = lib.rascal_neighbours_noalloc(calc._ctx, C.byref(sys_c), capacity, C.c_void_p(off.data_ptr()),
                                       C.c_void_p(nbr.data_ptr()), C.c_void_p(sh.data_ptr()), C.c_void_p(rij.data_ptr()),
                                       C.byref(P))
    rg._lib.check(st)
    n = P.value
    return off.cpu().numpy(), nbr[:n].cpu().numpy(), sh[:n].cpu().numpy(), rij[:n].cpu().numpy()


def _compare(rg, system):
    calc = rg.SoapCalculator(**system.hypers)
    ds = rg.DeviceSystem.from_numpy(system)
    ref = calc.neighbours(ds)
    got = _noalloc(rg, calc, ds, capacity=ref.n_pairs + 7)
    assert np.array_equal(got[0], ref.offsets.cpu().numpy())
    assert np.array_equal(got[1], ref.nbr_j.cpu().numpy())
    assert np.array_equal(got[2], ref.shifts.cpu().numpy())
    assert np.array_equal(got[3], ref.rij.cpu().numpy())
    return got


def test_two_calls_in_a_row_match_the_allocating_entry_point(rg):
    first = _compare(rg, config_batch(n_structures=64))
    second = _compare(rg, small_cell_system(seed=12, n_atoms=7, L=4.0))  # reuses the array left by the first call
    assert len(first[1]) > len(second[1]) > 0


def _dense_cell(density, n_seed, d_min, L=16.0, r_cut=7.0):
    """One cubic cell dense enough that every centre has well over 128 neighbours within r_cut."""
    n = int(round(density * L ** 3))
    rng = np.random.Generator(np.random.PCG64(n_seed))
    pos = random_cell_atoms(n, np.eye(3) * L, d_min, rng)
    return System(pos, np.full(n, 6, np.int32), (np.eye(3) * L)[None], np.ones((1, 3), np.int32),
                  np.array([0, n], np.int32), dict(r_cut=r_cut, sigma=0.5, n_max=2, l_max=1, smooth_width=0.5, species=[6]))


def test_centres_with_129_to_256_neighbours_match_the_allocating_entry_point(rg):
    # 532 atoms, 164..202 neighbours per centre: the no-allocation sort uses all of its lanes here, while
    # rascal_neighbours takes its overflow path for every centre
    s = _dense_cell(0.13, 51, 1.2)
    off, nbr, _, _ = _compare(rg, s)
    counts = np.diff(off)
    assert counts.min() > 128 and counts.max() <= 256


def test_centres_above_256_neighbours_are_refused_before_the_capacity_check(rg):
    import torch

    s = _dense_cell(0.25, 52, 1.0)  # 1024 atoms, 336..379 neighbours per centre
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    lib = rg._lib.lib()
    off = torch.empty(s.n_atoms + 1, dtype=torch.int64, device="cuda")
    P = C.c_int64(0)
    calc._bind_stream()
    sys_c = ds.c_struct()
    st = lib.rascal_neighbours_noalloc(calc._ctx, C.byref(sys_c), 0, C.c_void_p(off.data_ptr()), None, None, None,
                                       C.byref(P))
    assert st == rg._lib.RASCAL_E_UNSUPPORTED, st
    assert b"neighbours" in lib.rascal_last_error()
    ref = calc.neighbours(ds)
    assert P.value == ref.n_pairs  # the counting pass ran and reported the pair count
    _compare(rg, config_tiny())


def test_sizes_beyond_the_array_are_refused_before_running(rg):
    import torch

    lib = rg._lib.lib()
    limit = lib.rascal_neighbours_static_limit()
    assert limit == 32 << 20
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    # a system whose atom count needs more scratch than the array. Every buffer is sized for all n_big atoms and
    # kept alive for the whole call, so even if the size check were to let it through, the kernels would only read
    # memory that exists
    n_big = int(limit // 100)
    rng = np.random.default_rng(3)
    L = 400.0
    pos = torch.tensor(rng.uniform(0.0, L, (n_big, 3)), dtype=torch.float64, device="cuda")
    species = torch.full((n_big,), 14, dtype=torch.int32, device="cuda")
    struct_off = torch.tensor([0, n_big], dtype=torch.int32, device="cuda")
    cell = (torch.eye(3, dtype=torch.float64, device="cuda") * L).contiguous()
    pbc = torch.ones((1, 3), dtype=torch.int32, device="cuda")
    off = torch.empty(n_big + 1, dtype=torch.int64, device="cuda")
    sys_c = rg._lib.System(1, n_big, struct_off.data_ptr(), pos.data_ptr(), cell.data_ptr(), pbc.data_ptr(),
                           species.data_ptr())
    P = C.c_int64(0)
    calc._bind_stream()
    st = lib.rascal_neighbours_noalloc(calc._ctx, C.byref(sys_c), 0, C.c_void_p(off.data_ptr()), None, None, None, C.byref(P))
    torch.cuda.synchronize()
    assert st == rg._lib.RASCAL_E_UNSUPPORTED
    assert b"no-allocation" in lib.rascal_last_error()
    # the context is untouched and keeps working
    _compare(rg, s)


def test_no_scratch_is_allocated_by_the_call(rg):
    # a fresh context: the call leaves the context's scratch arenas exactly as rascal_create left them
    s = config_batch(n_structures=16)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    before = calc.scratch_bytes()
    got = _noalloc(rg, calc, ds, capacity=64 * s.n_atoms)
    calc.sync()
    assert calc.scratch_bytes() == before
    assert got[0][-1] > 0
