"""Failure paths of the tensor-core kernels, made without faulting the GPU.

The persistent fused kernel's mbarrier waits are bounded. rascal_set_wait_limit (a test hook) lowers the bound to a
single poll, so the first wait for an MMA batch runs out: the kernel must raise the timeout flag, leave every loop,
drain the MMAs already issued with the full bound and free its tensor memory; the next synchronising call returns
RASCAL_E_TIMEOUT and the same context then computes correct results again.
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


@pytest.mark.parametrize("precision", ["tf32x3", "bf16"])
def test_bounded_wait_times_out_and_the_context_recovers(rg, precision):
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    lib = rg._lib.lib()
    assert lib.rascal_set_wait_limit(calc._ctx, 1) == rg._lib.RASCAL_OK
    calc.soap(ds, pairs, precision=precision)
    with pytest.raises(rg.RascalError) as e:
        calc.sync()
    assert e.value.code == rg._lib.RASCAL_E_TIMEOUT
    assert lib.rascal_set_wait_limit(calc._ctx, 0) == rg._lib.RASCAL_OK
    c, p = calc.soap(ds, pairs, precision=precision)
    calc.sync()
    h = osoap.Hypers(**s.hypers)
    c_ref = osoap.spherical_expansion(s, h)
    p_ref = osoap.power_spectrum(c_ref, h, "packed")
    assert block_rel_err(c.cpu().numpy(), c_ref, 2) <= 1e-5
    err = block_rel_err(ps_blocks(p.cpu().numpy(), h.l_max), p_ref.reshape(s.n_atoms, h.l_max + 1, -1), 2)
    assert err <= (1e-5 if precision == "tf32x3" else 2.0 ** -7), err
