"""GPU nu = 2 equivariants (lambda-SOAP) against the FP64 oracle.

Tolerance (FP32 path): per (centre, pair) block of T, max |gpu - oracle| / max |oracle| <= 1e-5, as for p (T is the
same kind of product of two coefficients); from the oracle's own coefficients rounded to FP32, 2e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lambda_soap as ols  # noqa: E402
from oracle import soap as osoap  # noqa: E402
from synth import config_tiny, small_cell_system  # noqa: E402
from tests.gpu_common import block_rel_err  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _gpu_c(rg, s, **over):
    calc = rg.SoapCalculator(**dict(s.hypers, **over))
    ds = rg.DeviceSystem.from_numpy(s)
    c = calc.spherical_expansion(ds, calc.neighbours(ds))
    return calc, c


@pytest.mark.parametrize("lam", [0, 1, 2, 3])
def test_tiny_against_oracle(rg, lam):
    s = config_tiny()
    h = osoap.Hypers(**s.hypers)
    calc, c = _gpu_c(rg, s)
    T = calc.lambda_soap(c, lam)
    calc.sync()
    c_ref = osoap.spherical_expansion(s, h)
    T_ref = ols.equivariants(c_ref, h, lam)
    assert T.shape == T_ref.shape and calc.lambda_soap_size(lam) == (T_ref.shape[1], int(np.prod(T_ref.shape[1:])))
    assert block_rel_err(T.cpu().numpy(), T_ref, 2) <= 1e-5


def test_from_the_oracles_coefficients(rg):
    import torch

    s = config_tiny()
    h = osoap.Hypers(**s.hypers)
    calc = rg.SoapCalculator(**s.hypers)
    c32 = osoap.spherical_expansion(s, h, centres=np.arange(20)).astype(np.float32)
    T = calc.lambda_soap(torch.tensor(c32, device=calc.device), 2)
    calc.sync()
    T_ref = ols.equivariants(c32.astype(np.float64), h, 2)
    assert block_rel_err(T.cpu().numpy(), T_ref, 2) <= 2e-6


@pytest.mark.parametrize("n_max,species,lam", [(6, [1, 8], 2), (3, [1], 1), (3, [1], 4)])
def test_small_cell_vector_and_scalar_stores(rg, n_max, species, lam):
    """Q = 12 (16-byte stores) and Q = 3 (scalar stores); lambda = 4 at l_max = 2 is the top rank (one pair)."""
    l_max = 5 if lam < 4 else 2
    s = small_cell_system(seed=27, n_atoms=8, L=4.9, hypers=dict(r_cut=4.5, sigma=0.5, n_max=n_max, l_max=l_max,
                                                                 smooth_width=0.6, species=species))
    h = osoap.Hypers(**s.hypers)
    calc, c = _gpu_c(rg, s)
    T = calc.lambda_soap(c, lam)
    calc.sync()
    T_ref = ols.equivariants(osoap.spherical_expansion(s, h), h, lam)
    assert block_rel_err(T.cpu().numpy(), T_ref, 2) <= 1e-5


def test_lambda_zero_is_signed_power_spectrum_on_the_gpu(rg):
    s = config_tiny()
    calc, c = _gpu_c(rg, s)
    T = calc.lambda_soap(c, 0).cpu().numpy()
    p = calc.power_spectrum(c, layout="full").cpu().numpy().reshape(s.n_atoms, calc.l_max + 1, 8, 8)
    for l in range(calc.l_max + 1):
        assert np.allclose(T[:, l, 0], (-1) ** l * p[:, l], rtol=1e-5, atol=1e-6 * np.max(np.abs(p[:, l])))


def test_lambda_range(rg):
    s = config_tiny()
    calc, c = _gpu_c(rg, s)
    with pytest.raises(rg.RascalError):
        calc.lambda_soap_size(2 * calc.l_max + 1)
    with pytest.raises(rg.RascalError):
        calc.lambda_soap(c, -1)
    n_pairs, _ = calc.lambda_soap_size(2 * calc.l_max)
    assert n_pairs == 1


def test_no_centres_and_isolated_atoms(rg):
    import torch

    from synth import System

    pos = np.array([[1.0, 1.0, 1.0], [9.0, 9.0, 9.0]])
    s = System(pos, np.array([14, 14], np.int32), np.eye(3)[None] * 30.0, np.ones((1, 3), np.int32),
               np.array([0, 2], np.int32), dict(r_cut=5.0, sigma=0.5, n_max=2, l_max=2, smooth_width=0.5, species=[14]))
    calc, c = _gpu_c(rg, s)
    T = calc.lambda_soap(c, 2)
    assert np.all(T.cpu().numpy() == 0.0)
    T0 = calc.lambda_soap(torch.zeros((0, 1, 2, 9), device=calc.device), 1)
    calc.sync()
    assert T0.shape[0] == 0


def test_batch_full_size_sampled(rg):
    """The bench's configuration: batch workload, c from the expansion kernel, rank 1 (17.8 GB of output)."""
    import torch

    from synth import config_batch

    s = config_batch()
    h = osoap.Hypers(**s.hypers)
    calc, c = _gpu_c(rg, s)
    T = calc.lambda_soap(c, 1)
    rng = np.random.default_rng(4)
    centres = np.concatenate([[0, s.n_atoms - 1], rng.choice(s.n_atoms, 10, replace=False)])
    Ts = T[torch.as_tensor(centres, device=T.device)].cpu().numpy()
    calc.sync()
    del T
    T_ref = ols.equivariants(osoap.spherical_expansion(s, h, centres=centres), h, 1)
    assert block_rel_err(Ts, T_ref, 2) <= 1e-5
