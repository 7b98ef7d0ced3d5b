"""tcgen05 power spectrum (BF16 and TF32x3) against the FP64 Gram of the oracle's coefficients.

Tolerances per (centre, l) block:
* TF32x3 and FP32: max |gpu - oracle| / max |oracle| <= 1e-5 (the hi/lo split leaves about 2^-21 per product);
* BF16 inputs: bfloat16 has 8 significant bits, unit roundoff u = 2^-8, so a product of two rounded inputs is off by
  up to 2u = 2^-7 relative; the block max-relative error is held to 2^-7 and the block's relative Frobenius-norm
  error ||dp|| / ||p|| to the 5e-3 target (the FP64 Gram of bf16-rounded inputs reaches 4.6e-3 on these workloads).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import soap as osoap  # noqa: E402
from synth import System, config_batch, config_tiny, random_cell_atoms  # noqa: E402
from tests.gpu_common import block_rel_err, ps_blocks  # noqa: E402

TOL = {"bf16": 5e-3, "tf32x3": 1e-5, "fp32": 1e-5}


@pytest.fixture(scope="module")
def rg():
    import paper_2101_08814_gb300 as rg

    return rg


def _system(n_species, n_max, l_max, r_cut=5.0, n_atoms=160, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (n_atoms / 0.05) ** (1 / 3)
    pos = random_cell_atoms(n_atoms, np.eye(3) * L, 1.6, rng)
    labels = list(range(1, n_species + 1))
    spe = np.asarray(labels, np.int32)[rng.integers(0, n_species, n_atoms)]
    return System(pos, spe, (np.eye(3) * L)[None], np.ones((1, 3), np.int32), np.array([0, n_atoms], np.int32),
                  dict(r_cut=r_cut, sigma=0.5, n_max=n_max, l_max=l_max, smooth_width=0.5, species=labels))


def _check(rg, s, layouts=("packed", "full"), centres=None):
    """Separate power spectrum from the oracle's own coefficients (rounded to FP32) against the FP64 Gram of exactly
    those inputs; fused power spectrum (c from the GPU's pair kernel) against the oracle's p at the same per-block
    bar (1e-5 for FP32 and TF32x3)."""
    import torch

    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    c = calc.spherical_expansion(ds, pairs)
    h = osoap.Hypers(**s.hypers)
    sel = np.arange(s.n_atoms) if centres is None else np.asarray(centres)
    c_ref = osoap.spherical_expansion(s, h, centres=sel)
    c32 = c_ref.astype(np.float32)
    c32_dev = torch.tensor(c32, device=calc.device)
    for layout in layouts:
        ref32 = osoap.power_spectrum(c32.astype(np.float64), h, layout)
        ref = osoap.power_spectrum(c_ref, h, layout)
        for prec, fused in [(p_, f_) for p_ in ("bf16", "tf32x3", "fp32") for f_ in (False, True)]:
            try:
                if fused:
                    c2, p = calc.soap(ds, pairs, layout=layout, precision=prec)
                    calc.sync()
                    if prec == "fp32":  # the same pair kernel as rascal_spherical_expansion
                        assert np.array_equal(c2.cpu().numpy(), c.cpu().numpy())
                    else:  # the persistent tensor-core kernel has its own pair phase (f_cut folded into Y_lm)
                        assert block_rel_err(c2.cpu().numpy()[sel], c_ref, 2) <= 1e-5
                    got, r, tol = p.cpu().numpy()[sel], ref, TOL[prec]
                else:
                    p = calc.power_spectrum(c32_dev, precision=prec, layout=layout)
                    calc.sync()
                    got, r, tol = p.cpu().numpy(), ref32, TOL[prec]
            except rg.RascalError as e:
                # the TF32 hi/lo operand tiles of n_species*n_max = 128, l_max = 12 exceed shared memory: the
                # library refuses them with RASCAL_E_UNSUPPORTED instead of running
                assert e.code == rg._lib.RASCAL_E_UNSUPPORTED and prec == "tf32x3" and h.q > 96, (prec, fused, str(e))
                continue
            gb, rb = ps_blocks(got, h.l_max), r.reshape(len(sel), h.l_max + 1, -1)
            err = block_rel_err(gb, rb, 2)
            if prec == "bf16":
                assert err <= 2.0 ** -7, (layout, prec, fused, err)
                fro = np.sqrt(np.sum((gb - rb) ** 2, axis=-1) / np.maximum(np.sum(rb ** 2, axis=-1), 1e-300))
                assert np.max(fro) <= 5e-3, (layout, prec, fused, np.max(fro))
            else:
                assert err <= tol, (layout, prec, fused, err)
            assert np.all(np.isfinite(got))


def test_tiny_single_species(rg):
    _check(rg, config_tiny())


def test_q30_needs_padded_columns(rg):
    _check(rg, _system(3, 10, 8, r_cut=6.0))


def test_q128_many_l_groups(rg):
    _check(rg, _system(8, 16, 12, r_cut=6.0, n_atoms=120), centres=[0, 50, 119])


def test_batch_full_size_sampled(rg):
    s = config_batch()
    rng = np.random.default_rng(2)
    _check(rg, s, layouts=("packed",), centres=np.concatenate([[0, s.n_atoms - 1], rng.choice(s.n_atoms, 30, replace=False)]))


def test_isolated_atoms_and_crowded_centres(rg):
    # a dense cluster (centres with more neighbours than one staged chunk) next to atoms with no neighbour at all:
    # the isolated centres' c and p are exactly zero in every form, the crowded ones match the oracle
    rng = np.random.Generator(np.random.PCG64(17))
    L = 40.0
    cluster = random_cell_atoms(70, np.eye(3) * 9.0, 1.05, rng) + 4.0
    lone = np.array([[30.0, 30.0, 30.0], [30.0, 8.0, 30.0], [8.0, 30.0, 20.0]])
    pos = np.concatenate([cluster, lone])
    spe = np.where(rng.random(len(pos)) < 0.5, 1, 8).astype(np.int32)
    s = System(pos, spe, (np.eye(3) * L)[None], np.zeros((1, 3), np.int32), np.array([0, len(pos)], np.int32),
               dict(r_cut=5.0, sigma=0.5, n_max=6, l_max=5, smooth_width=0.5, species=[1, 8]))
    calc = rg.SoapCalculator(**s.hypers)
    ds = rg.DeviceSystem.from_numpy(s)
    pairs = calc.neighbours(ds)
    counts = np.diff(pairs.offsets.cpu().numpy())
    assert counts.max() > 32 and np.all(counts[-3:] == 0)
    _check(rg, s)
    for prec in ("fp32", "bf16", "tf32x3"):
        c, p = calc.soap(ds, pairs, precision=prec)
        calc.sync()
        assert np.all(c.cpu().numpy()[-3:] == 0.0) and np.all(p.cpu().numpy()[-3:] == 0.0), prec
