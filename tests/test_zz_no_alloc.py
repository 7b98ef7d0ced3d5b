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

from synth import config_batch, config_tiny, small_cell_system  # noqa: E402


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


def test_sizes_beyond_the_array_are_refused_before_running(rg):
    import torch

    lib = rg._lib.lib()
    limit = lib.rascal_neighbours_static_limit()
    assert limit == 32 << 20
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    # a system description whose atom count needs more scratch than the array; nothing is launched, so the
    # device arrays only need to exist
    n_big = int(limit // 100)
    pos = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    sys_c = rg._lib.System(1, n_big, torch.tensor([0, n_big], dtype=torch.int32, device="cuda").data_ptr(), pos.data_ptr(),
                           torch.eye(3, dtype=torch.float64, device="cuda").data_ptr(), 0,
                           torch.zeros(1, dtype=torch.int32, device="cuda").data_ptr())
    off = torch.empty(4, dtype=torch.int64, device="cuda")
    P = C.c_int64(0)
    st = lib.rascal_neighbours_noalloc(calc._ctx, C.byref(sys_c), 0, C.c_void_p(off.data_ptr()), None, None, None, C.byref(P))
    assert st == rg._lib.RASCAL_E_UNSUPPORTED
    assert b"no-allocation" in lib.rascal_last_error()
    # the context is untouched and keeps working
    _compare(rg, s)
