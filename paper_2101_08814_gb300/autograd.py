"""torch.autograd wrappers around the library's forward and backward kernels (argument marshalling only).

PowerSpectrumFunction: positions -> PACKED power spectrum p [N, F]; its backward receives dL/dp and returns
dL/dpositions = -F computed by rascal_gradients (per-pair recomputation, no stored dc/dr).
LinearSoapEnergy: the additive linear model E_s = sum_{i in s} w_{a_i} . p_i, with forces and virial from the
backward kernel in one call.
"""
from __future__ import annotations

import torch

from . import DeviceSystem, SoapCalculator


class PowerSpectrumFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, positions, calc: SoapCalculator, system: DeviceSystem):
        ds = DeviceSystem(positions.detach().contiguous(), system.species, system.cells, system.pbc, system.struct_offsets)
        pairs = calc.neighbours(ds)
        coeffs, ps = calc.soap(ds, pairs, layout="packed")
        ctx.calc, ctx.ds, ctx.pairs = calc, ds, pairs
        ctx.save_for_backward(coeffs)
        return ps

    @staticmethod
    def backward(ctx, grad_ps):
        (coeffs,) = ctx.saved_tensors
        forces, _ = ctx.calc.gradients(ctx.ds, ctx.pairs, coeffs, grad_ps=grad_ps.contiguous().float())
        return -forces.to(grad_ps.dtype if grad_ps.dtype == torch.float64 else torch.float64), None, None


def power_spectrum(positions, calc: SoapCalculator, system: DeviceSystem):
    return PowerSpectrumFunction.apply(positions, calc, system)


class LinearSoapEnergy:
    """E = sum_i w_{a_i} . p_i per structure, with analytic forces F = -dE/dr and virial sum_ij dE/dr_ji (x) r_ji."""

    def __init__(self, calc: SoapCalculator, weights: torch.Tensor):
        self.calc = calc
        self.weights = weights.to(device=calc.device, dtype=torch.float32).contiguous()

    def __call__(self, system: DeviceSystem, forces=True):
        pairs = self.calc.neighbours(system)
        coeffs, ps = self.calc.soap(system, pairs, layout="packed")
        energy = self.calc.linear_energy(system, ps, self.weights)
        if not forces:
            return energy, None, None
        f, v = self.calc.gradients(system, pairs, coeffs, weights=self.weights)
        return energy, f, v
