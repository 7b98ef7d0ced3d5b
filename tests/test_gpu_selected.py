"""Selected power-spectrum features (sparse feature selection) from the fused kernel against the oracle.

The oracle's packed power spectrum, indexed by the selection, is the definition; tolerance as for the FP32 path:
per (centre) row of selected features, max |gpu - oracle| / max |oracle| <= 1e-5.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import soap as osoap  # noqa: E402
from synth import System, config_tiny, random_cell_atoms  # noqa: E402
from tests.gpu_common import block_rel_err  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _system(seed=5, n_atoms=150):
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (n_atoms / 0.05) ** (1 / 3)
    pos = random_cell_atoms(n_atoms, np.eye(3) * L, 1.6, rng)
    spe = np.asarray([1, 6, 8], np.int32)[rng.integers(0, 3, n_atoms)]
    return System(pos, spe, (np.eye(3) * L)[None], np.ones((1, 3), np.int32), np.array([0, n_atoms], np.int32),
                  dict(r_cut=5.0, sigma=0.5, n_max=5, l_max=6, smooth_width=0.5, species=[1, 6, 8]))


@pytest.mark.parametrize("make", [config_tiny, _system])
def test_selected_features_match_oracle(rg, make):
    s = make()
    h = osoap.Hypers(**s.hypers)
    F = h.n_features("packed")
    rng = np.random.default_rng(3)
    sel = np.concatenate([[0, F - 1], rng.choice(F, size=max(3, F // 10), replace=False), [7, 7]]).astype(np.int32)
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c, p = calc.soap_selected(ds, pairs, sel)
    c_full, p_full = calc.soap(ds, pairs)
    calc.sync()
    assert np.array_equal(c.cpu().numpy(), c_full.cpu().numpy())
    ref = osoap.power_spectrum(osoap.spherical_expansion(s, h), h, "packed").reshape(s.n_atoms, -1)[:, sel]
    assert block_rel_err(p.cpu().numpy(), ref, 1) <= 1e-5
    assert np.array_equal(p.cpu().numpy()[:, -2], p.cpu().numpy()[:, -1])  # a repeated index gives the same column


def test_out_of_range_index_is_refused(rg):
    s = config_tiny()
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    F = calc.n_features("packed")
    with pytest.raises(rg.RascalError) as e:
        calc.soap_selected(ds, pairs, np.array([0, F], np.int32))
        calc.sync()
    assert e.value.code == rg._lib.RASCAL_E_ARG
    calc.sync()  # the flag is cleared once reported
