"""GB300 (sm_103a) SOAP density expansion of arXiv:2101.08814 behind a C ABI (include/rascal.h).

This module is the thin Python binding: it allocates output tensors with PyTorch, passes device pointers and the
current CUDA stream to the library, and turns status codes into exceptions. Every step of the computation runs
in the library's CUDA kernels; there is no CPU path. Importing works without a GPU; creating a calculator needs
the built library and a CUDA device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

from . import _lib
from ._lib import LAYOUT, PRECISION, RADIAL, RascalError  # noqa: F401


def _ptr(t):
    """Device address of a tensor. An empty view (e.g. the pair arrays of a system without pairs) reports 0 from
    data_ptr(); its storage address is passed instead, so that the library's NULL checks only reject missing buffers."""
    if t is None:
        return C.c_void_p(0)
    p = t.data_ptr()
    if p == 0 and t.numel() == 0:
        p = t.untyped_storage().data_ptr()
    return C.c_void_p(p)


def _need(t, numel: int, what: str):
    """A caller-provided buffer must be a contiguous float32 tensor with room for `numel` values: the library writes
    through raw pointers and cannot check sizes itself."""
    import torch

    if t is None:
        return t
    if t.dtype != torch.float32 or not t.is_contiguous() or t.device.type != "cuda" or t.numel() < numel:
        raise ValueError(f"{what}: need a contiguous float32 CUDA tensor of at least {numel} values, got "
                         f"{tuple(t.shape)} {t.dtype} on {t.device}")
    return t


def launch_count() -> int:
    """Kernels the library has launched in this process (all contexts)."""
    return int(_lib.lib().rascal_launch_count())


@dataclass
class DeviceSystem:
    """Structures resident on the GPU (tensors kept alive for the duration of the calls)."""

    positions: "object"       # torch.float64 [N, 3]
    species: "object"         # torch.int32 [N]
    cells: "object"           # torch.float64 [n_s, 3, 3]
    pbc: "object"             # torch.int32 [n_s, 3]
    struct_offsets: "object"  # torch.int32 [n_s + 1]

    @property
    def n_atoms(self):
        return int(self.positions.shape[0])

    @property
    def n_structures(self):
        return int(self.cells.shape[0])

    def c_struct(self):
        return _lib.System(self.n_structures, self.n_atoms, self.struct_offsets.data_ptr(), self.positions.data_ptr(),
                           self.cells.data_ptr(), self.pbc.data_ptr(), self.species.data_ptr())

    @staticmethod
    def from_numpy(system, device="cuda"):
        import torch

        return DeviceSystem(
            torch.as_tensor(system.positions, dtype=torch.float64, device=device).contiguous(),
            torch.as_tensor(system.species, dtype=torch.int32, device=device).contiguous(),
            torch.as_tensor(system.cells, dtype=torch.float64, device=device).contiguous(),
            torch.as_tensor(system.pbc, dtype=torch.int32, device=device).contiguous(),
            torch.as_tensor(system.struct_offsets, dtype=torch.int32, device=device).contiguous(),
        )


@dataclass
class PairList:
    offsets: "object"  # int64 [N+1]
    nbr_j: "object"    # int32 [P]
    shifts: "object"   # int32 [P, 3]
    rij: "object"      # float32 [P, 4] (x, y, z, r)

    @property
    def n_pairs(self):
        return int(self.nbr_j.shape[0])


class SoapCalculator:
    """Owns one library context (radial spline table and scratch) for a set of hypers."""

    def __init__(self, r_cut, sigma, n_max, l_max, species, smooth_width=0.5, radial="spline", orthonormal=True,
                 include_center=False, ps_norm=True, spline_accuracy=0.0, spline_intervals=0, basis="gto", device=None,
                 **_ignored):
        import torch

        self.device = torch.device("cuda" if device is None else device)
        self.species = sorted(int(s) for s in species)
        arr = (C.c_int * len(self.species))(*self.species)
        self._species_arr = arr
        h = _lib.Hypers(float(r_cut), float(smooth_width), float(sigma), int(n_max), int(l_max), len(self.species),
                        C.cast(arr, C.POINTER(C.c_int)), RADIAL[radial], int(bool(orthonormal)), int(bool(include_center)),
                        int(bool(ps_norm)), float(spline_accuracy), int(spline_intervals), _lib.BASIS[basis])
        self._ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream().cuda_stream
            _lib.check(_lib.lib().rascal_create(C.byref(h), C.c_void_p(stream), C.byref(self._ctx)))
        info = _lib.Info()
        _lib.check(_lib.lib().rascal_info(self._ctx, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in _lib.Info._fields_}
        self.n_max, self.l_max, self.n_species = int(n_max), int(l_max), len(self.species)
        self._capacity = 0

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx is not None and ctx.value:
            try:
                _lib.lib().rascal_destroy(ctx)
            except Exception:
                pass
            self._ctx = None

    # ----------------------------------------------------------------------------------------------------------
    def _bind_stream(self):
        import torch

        _lib.check(_lib.lib().rascal_set_stream(self._ctx, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))

    @property
    def coeffs_per_centre(self):
        return int(self.info["coeffs_per_centre"])

    def n_features(self, layout="packed"):
        return int(self.info["features_packed" if layout == "packed" else "features_full"])

    def scratch_bytes(self):
        """Device bytes the context's scratch arenas hold now (they grow on demand and are kept)."""
        info = _lib.Info()
        _lib.check(_lib.lib().rascal_info(self._ctx, C.byref(info)))
        return int(info.scratch_bytes)

    def sync(self):
        self._bind_stream()
        _lib.check(_lib.lib().rascal_sync(self._ctx))

    def neighbours(self, system: DeviceSystem, capacity=None) -> PairList:
        import torch

        self._bind_stream()
        N = system.n_atoms
        offsets = torch.empty(N + 1, dtype=torch.int64, device=self.device)
        cap = int(capacity if capacity is not None else max(self._capacity, 64 * N, 1))
        sys_c = system.c_struct()
        while True:
            nbr = torch.empty(cap, dtype=torch.int32, device=self.device)
            shifts = torch.empty((cap, 3), dtype=torch.int32, device=self.device)
            rij = torch.empty((cap, 4), dtype=torch.float32, device=self.device)
            P = C.c_int64(0)
            st = _lib.lib().rascal_neighbours(self._ctx, C.byref(sys_c), cap, _ptr(offsets), _ptr(nbr), _ptr(shifts),
                                              _ptr(rij), C.byref(P))
            if st == _lib.RASCAL_E_CAPACITY:
                cap = int(P.value * 1.1) + 16
                continue
            _lib.check(st)
            break
        self._capacity = max(self._capacity, cap)
        n = int(P.value)
        return PairList(offsets, nbr[:n], shifts[:n], rij[:n])

    def spherical_expansion(self, system: DeviceSystem, pairs: PairList, out=None):
        import torch

        self._bind_stream()
        N = system.n_atoms
        c = _need(out, N * self.coeffs_per_centre, "out") if out is not None else \
            torch.empty((N, self.n_species, self.n_max, (self.l_max + 1) ** 2), dtype=torch.float32, device=self.device)
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_spherical_expansion(self._ctx, C.byref(sys_c), _ptr(pairs.offsets),
                                                         _ptr(pairs.nbr_j), _ptr(pairs.rij), _ptr(c)))
        return c

    def power_spectrum(self, coeffs, precision="fp32", layout="packed", out=None):
        import torch

        self._bind_stream()
        n = int(coeffs.shape[0])
        _need(coeffs, n * self.coeffs_per_centre, "coeffs")
        p = _need(out, n * self.n_features(layout), "out") if out is not None else \
            torch.empty((n, self.n_features(layout)), dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().rascal_power_spectrum(self._ctx, n, _ptr(coeffs), PRECISION[precision], LAYOUT[layout],
                                                    _ptr(p)))
        return p

    def soap(self, system: DeviceSystem, pairs: PairList, layout="packed", precision="fp32", coeffs=None, ps=None):
        """Expansion and power spectrum in one fused kernel launch."""
        import torch

        self._bind_stream()
        N = system.n_atoms
        c = _need(coeffs, N * self.coeffs_per_centre, "coeffs") if coeffs is not None else \
            torch.empty((N, self.n_species, self.n_max, (self.l_max + 1) ** 2), dtype=torch.float32, device=self.device)
        p = _need(ps, N * self.n_features(layout), "ps") if ps is not None else \
            torch.empty((N, self.n_features(layout)), dtype=torch.float32, device=self.device)
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_soap(self._ctx, C.byref(sys_c), _ptr(pairs.offsets), _ptr(pairs.nbr_j),
                                          _ptr(pairs.rij), PRECISION[precision], LAYOUT[layout], _ptr(c), _ptr(p)))
        return c, p

    def soap_selected(self, system: DeviceSystem, pairs: PairList, sel, coeffs=None, ps=None):
        """c and the selected PACKED power-spectrum features ([N][len(sel)]) in one fused kernel launch."""
        import torch

        self._bind_stream()
        N = system.n_atoms
        sel = torch.as_tensor(sel, dtype=torch.int32, device=self.device).contiguous()
        c = _need(coeffs, N * self.coeffs_per_centre, "coeffs") if coeffs is not None else \
            torch.empty((N, self.n_species, self.n_max, (self.l_max + 1) ** 2), dtype=torch.float32, device=self.device)
        p = _need(ps, N * sel.numel(), "ps") if ps is not None else \
            torch.empty((N, sel.numel()), dtype=torch.float32, device=self.device)
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_soap_selected(self._ctx, C.byref(sys_c), _ptr(pairs.offsets), _ptr(pairs.nbr_j),
                                                   _ptr(pairs.rij), int(sel.numel()), _ptr(sel), _ptr(c), _ptr(p)))
        return c, p

    def linear_energy(self, system: DeviceSystem, ps_packed, weights):
        import torch

        self._bind_stream()
        _need(ps_packed, system.n_atoms * self.n_features("packed"), "ps_packed")
        _need(weights, self.n_species * self.n_features("packed"), "weights")
        e = torch.empty(system.n_structures, dtype=torch.float64, device=self.device)
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_linear_energy(self._ctx, C.byref(sys_c), _ptr(ps_packed), _ptr(weights), _ptr(e)))
        return e

    def gradients(self, system: DeviceSystem, pairs: PairList, coeffs, grad_ps=None, weights=None):
        import torch

        self._bind_stream()
        N = system.n_atoms
        _need(coeffs, N * self.coeffs_per_centre, "coeffs")
        _need(grad_ps, N * self.n_features("packed"), "grad_ps")
        _need(weights, self.n_species * self.n_features("packed"), "weights")
        forces = torch.empty((system.n_atoms, 3), dtype=torch.float64, device=self.device)
        virial = torch.empty((system.n_structures, 3, 3), dtype=torch.float64, device=self.device)
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_gradients(self._ctx, C.byref(sys_c), _ptr(pairs.offsets), _ptr(pairs.nbr_j),
                                               _ptr(pairs.rij), _ptr(coeffs), _ptr(grad_ps), _ptr(weights),
                                               _ptr(forces), _ptr(virial)))
        return forces, virial

    def debug_pair_gradients(self, rij):
        """d/dr_ji of each pair's term f_cut I^o_nl Y_lm: [P, 3, n_max, (l_max+1)^2] float32 (a test hook)."""
        import torch

        self._bind_stream()
        rij = rij.contiguous()
        if rij.dtype != torch.float32 or rij.dim() != 2 or rij.shape[1] != 4 or rij.device.type != "cuda":
            raise ValueError("rij must be a float32 [P, 4] CUDA tensor (x, y, z, r)")
        P = int(rij.shape[0])
        out = torch.empty((P, 3, self.n_max, (self.l_max + 1) ** 2), dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().rascal_debug_pair_gradients(self._ctx, P, _ptr(rij), _ptr(out)))
        return out

    def lambda_soap_size(self, lam: int):
        """(number of (l1, l2) pairs, features per centre) of the rank-lam equivariants."""
        n_pairs, feat = C.c_int(), C.c_int64()
        _lib.check(_lib.lib().rascal_lambda_soap_size(self._ctx, int(lam), C.byref(n_pairs), C.byref(feat)))
        return n_pairs.value, feat.value

    def lambda_soap(self, coeffs, lam: int, out=None):
        """nu = 2 equivariants of rank lam: [N, n_pairs, 2 lam + 1, Q, Q] float32 from c [N, S, n_max, n_lm]."""
        import torch

        self._bind_stream()
        n_pairs, _ = self.lambda_soap_size(lam)
        N = coeffs.shape[0]
        Q = self.n_species * self.n_max
        _need(coeffs, N * self.coeffs_per_centre, "coeffs")
        o = _need(out, N * n_pairs * (2 * lam + 1) * Q * Q, "out") if out is not None else \
            torch.empty((N, n_pairs, 2 * lam + 1, Q, Q), dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().rascal_lambda_soap(self._ctx, N, _ptr(coeffs), int(lam), _ptr(o)))
        return o

    # ---------------------------------------------------------------------------------------- radial source
    def set_radial(self, mode: str):
        """'spline' (table), 'exact' (per-pair 1F1 in FP64) or 'mlp' (the trained network)."""
        _lib.check(_lib.lib().rascal_set_radial(self._ctx, RADIAL[mode]))

    # ---------------------------------------------------------------------------------------- MLP surrogate
    MLP_HIDDEN = 64

    def mlp_num_params(self):
        return int(_lib.lib().rascal_mlp_num_params(self._ctx, self.MLP_HIDDEN))

    def mlp_set_params(self, params, scale):
        import numpy as np

        p = np.ascontiguousarray(params, dtype=np.float32)
        s = np.ascontiguousarray(scale, dtype=np.float32)
        if p.size != self.mlp_num_params() or s.size != self.n_max * (self.l_max + 1):
            raise ValueError("parameter or scale vector of the wrong size")
        self._bind_stream()
        _lib.check(_lib.lib().rascal_mlp_set_params(self._ctx, self.MLP_HIDDEN, p.ctypes.data_as(C.c_void_p),
                                                    s.ctypes.data_as(C.c_void_p)))

    def mlp_get_params(self):
        import numpy as np

        p = np.empty(self.mlp_num_params(), dtype=np.float32)
        s = np.empty(self.n_max * (self.l_max + 1), dtype=np.float32)
        self._bind_stream()
        _lib.check(_lib.lib().rascal_mlp_get_params(self._ctx, p.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p)))
        return p, s

    def mlp_targets(self, r, dense_intervals=0):
        """Scaled FP64-exact targets [n, F] (float32, device) at distances r, and the scales [F] (numpy)."""
        import numpy as np
        import torch

        self._bind_stream()
        r = torch.as_tensor(r, dtype=torch.float64, device=self.device).contiguous()
        F = self.n_max * (self.l_max + 1)
        out = torch.empty((r.shape[0], F), dtype=torch.float32, device=self.device)
        scale = np.empty(F, dtype=np.float32)
        _lib.check(_lib.lib().rascal_mlp_targets(self._ctx, r.shape[0], _ptr(r), int(dense_intervals), _ptr(out),
                                                 scale.ctypes.data_as(C.c_void_p)))
        return out, scale

    def mlp_train(self, t, targets, order, batch, steps, lr_max=3e-3, lr_min=1e-5, total_steps=0, record_loss=True):
        import torch

        self._bind_stream()
        loss = torch.zeros(steps, dtype=torch.float32, device=self.device) if record_loss else None
        _lib.check(_lib.lib().rascal_mlp_train(self._ctx, int(t.shape[0]), _ptr(t), _ptr(targets), _ptr(order), int(batch),
                                               int(steps), float(lr_max), float(lr_min), int(total_steps), _ptr(loss)))
        return loss

    def mlp_gradients(self, t, targets):
        import torch

        self._bind_stream()
        g = torch.empty(self.mlp_num_params(), dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().rascal_mlp_gradients(self._ctx, int(t.shape[0]), _ptr(t), _ptr(targets), _ptr(g), _ptr(loss)))
        return g, loss

    def mlp_eval(self, r, derivative=False):
        import torch

        self._bind_stream()
        r = torch.as_tensor(r, dtype=torch.float32, device=self.device).contiguous()
        F = self.n_max * (self.l_max + 1)
        out = torch.empty((r.shape[0], F), dtype=torch.float32, device=self.device)
        dout = torch.empty_like(out) if derivative else None
        _lib.check(_lib.lib().rascal_mlp_eval(self._ctx, r.shape[0], _ptr(r), _ptr(out), _ptr(dout)))
        return (out, dout) if derivative else out

    def mlp_save(self, path):
        _lib.check(_lib.lib().rascal_mlp_save(self._ctx, str(path).encode()))

    def mlp_load(self, path):
        self._bind_stream()
        _lib.check(_lib.lib().rascal_mlp_load(self._ctx, str(path).encode()))

    def radial_exact_fp64(self, r, derivative=False):
        import torch

        self._bind_stream()
        r = r.to(device=self.device, dtype=torch.float64).contiguous()
        out = torch.empty((r.shape[0], self.n_max, self.l_max + 1), dtype=torch.float64, device=self.device)
        dout = torch.empty_like(out) if derivative else None
        _lib.check(_lib.lib().rascal_radial_exact_fp64(self._ctx, r.shape[0], _ptr(r), _ptr(out), _ptr(dout)))
        return (out, dout) if derivative else out


class GprModel:
    """Sparse GPR energy model with the polynomial kernel (Eq. sparse-gp), evaluated on the tensor cores.

    sparse [n_sparse, n_features] (host array), sparse_species [n_sparse] labels, weights [n_sparse] (x_I)."""

    def __init__(self, calc: SoapCalculator, sparse, sparse_species, weights, zeta=2, normalize=True):
        import numpy as np

        self.calc = calc
        sp = np.ascontiguousarray(sparse, dtype=np.float64)
        if sp.ndim != 2:
            raise ValueError("sparse points must be a 2-D array [n_sparse, n_features]")
        lab = np.ascontiguousarray(sparse_species, dtype=np.int32)
        x = np.ascontiguousarray(weights, dtype=np.float64)
        self.n_features = int(sp.shape[1])
        self.zeta, self.normalize = int(zeta), bool(normalize)
        self._h = C.c_void_p()
        _lib.check(_lib.lib().rascal_gpr_create(calc._ctx, sp.shape[0], sp.shape[1], sp.ctypes.data_as(C.c_void_p),
                                                lab.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p),
                                                self.zeta, int(self.normalize), C.byref(self._h)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.lib().rascal_gpr_destroy(h)
            except Exception:
                pass
            self._h = None

    def predict(self, system: DeviceSystem, features, grad=False, atomic=True):
        """(per-structure energies float64, per-centre energies float32 or None, dE/dp float32 or None)."""
        import torch

        calc = self.calc
        calc._bind_stream()
        e = torch.empty(system.n_structures, dtype=torch.float64, device=calc.device)
        ea = torch.empty(system.n_atoms, dtype=torch.float32, device=calc.device) if atomic else None
        g = torch.empty((system.n_atoms, self.n_features), dtype=torch.float32, device=calc.device) if grad else None
        f = features.reshape(system.n_atoms, self.n_features)
        if f.shape[1] != self.n_features or f.dtype != torch.float32 or not f.is_contiguous():
            raise ValueError("features must be a contiguous float32 [n_atoms, n_features] tensor")
        sys_c = system.c_struct()
        _lib.check(_lib.lib().rascal_gpr_predict(calc._ctx, self._h, C.byref(sys_c), _ptr(f), _ptr(ea), _ptr(e), _ptr(g)))
        return e, ea, g

