"""Failure paths of the tensor-core Gram, made without faulting the GPU.

Every MMA-completion wait of the fused kernel is bounded. The test hook rascal_debug_wait_timeout points the first
such wait of every CTA at an mbarrier that nothing arrives at, so it runs out for certain after the given number of
polls: the kernel must raise the timeout flag, skip the rest of its epilogues, wait for the MMAs it already issued
and free its tensor memory; the next synchronising call returns RASCAL_E_TIMEOUT and the same context then computes
correct results again.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import soap as osoap  # noqa: E402
from synth import config_tiny  # noqa: E402
from tests.gpu_common import block_rel_err, ps_blocks  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _check(s, c, p, precision):
    h = osoap.Hypers(**s.hypers)
    c_ref = osoap.spherical_expansion(s, h)
    p_ref = osoap.power_spectrum(c_ref, h, "packed")
    assert block_rel_err(c.cpu().numpy(), c_ref, 2) <= 1e-5
    err = block_rel_err(ps_blocks(p.cpu().numpy(), h.l_max), p_ref.reshape(s.n_atoms, h.l_max + 1, -1), 2)
    assert err <= (1e-5 if precision == "tf32x3" else 2.0 ** -7), err


@pytest.mark.parametrize("precision", ["tf32x3", "bf16"])
def test_bounded_wait_times_out_and_the_context_recovers(rg, precision):
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    lib = rg._lib.lib()
    assert lib.rascal_debug_wait_timeout(calc._ctx, 1000) == rg._lib.RASCAL_OK
    calc.soap(ds, pairs, precision=precision)
    with pytest.raises(rg.RascalError) as e:
        calc.sync()
    assert e.value.code == rg._lib.RASCAL_E_TIMEOUT
    # the separate tensor-core power spectrum runs the same Gram and takes the same path
    c = calc.spherical_expansion(ds, pairs)
    calc.power_spectrum(c, precision=precision)
    with pytest.raises(rg.RascalError) as e:
        calc.sync()
    assert e.value.code == rg._lib.RASCAL_E_TIMEOUT
    assert lib.rascal_debug_wait_timeout(calc._ctx, 0) == rg._lib.RASCAL_OK
    c, p = calc.soap(ds, pairs, precision=precision)
    calc.sync()
    _check(s, c, p, precision)
    p2 = calc.power_spectrum(c, precision=precision)
    calc.sync()
    _check(s, c, p2, precision)


def test_hook_refuses_a_null_context(rg):
    lib = rg._lib.lib()
    assert lib.rascal_debug_wait_timeout(None, 5) == rg._lib.RASCAL_E_ARG
