"""ctypes declarations of the C ABI in include/rascal.h. Loading fails loudly if the library was not built."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librascal_gb300.so")

RASCAL_OK = 0
RASCAL_E_ARG = -1
RASCAL_E_CAPACITY = -2
RASCAL_E_CUDA = -3
RASCAL_E_UNSUPPORTED = -4
RASCAL_E_GEOMETRY = -5
RASCAL_E_TIMEOUT = -6
RASCAL_E_NOMEM = -7

RADIAL = {"spline": 0, "exact": 1, "mlp": 2}
PRECISION = {"fp32": 0, "bf16": 1, "tf32x3": 2}
LAYOUT = {"packed": 0, "full": 1}
BASIS = {"gto": 0, "dvr": 1}


class Hypers(C.Structure):
    _fields_ = [
        ("r_cut", C.c_double),
        ("smooth_width", C.c_double),
        ("sigma", C.c_double),
        ("n_max", C.c_int),
        ("l_max", C.c_int),
        ("n_species", C.c_int),
        ("species", C.POINTER(C.c_int)),
        ("radial", C.c_int),
        ("orthonormal", C.c_int),
        ("include_center", C.c_int),
        ("ps_norm", C.c_int),
        ("spline_accuracy", C.c_double),
        ("spline_intervals", C.c_int),
        ("radial_basis", C.c_int),
    ]


class System(C.Structure):
    _fields_ = [
        ("n_structures", C.c_int),
        ("n_atoms", C.c_int),
        ("d_struct_offsets", C.c_void_p),
        ("d_positions", C.c_void_p),
        ("d_cells", C.c_void_p),
        ("d_pbc", C.c_void_p),
        ("d_species", C.c_void_p),
    ]


class Info(C.Structure):
    _fields_ = [
        ("n_species", C.c_int),
        ("n_max", C.c_int),
        ("l_max", C.c_int),
        ("n_lm", C.c_int),
        ("coeffs_per_centre", C.c_int64),
        ("features_packed", C.c_int64),
        ("features_full", C.c_int64),
        ("spline_intervals", C.c_int),
        ("spline_error", C.c_double),
        ("spline_error_fp32", C.c_double),
        ("scratch_bytes", C.c_int64),
    ]


class RascalError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"rascal error {code}: {message}")
        self.code = code


_lib = None

# name -> (restype, argtypes)
_SIGNATURES = {
    "rascal_last_error": (C.c_char_p, []),
    "rascal_launch_count": (C.c_longlong, []),
    "rascal_create": (C.c_int, [C.POINTER(Hypers), C.c_void_p, C.POINTER(C.c_void_p)]),
    "rascal_destroy": (None, [C.c_void_p]),
    "rascal_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rascal_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "rascal_sync": (C.c_int, [C.c_void_p]),
    "rascal_neighbours": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int64)]),
    "rascal_neighbours_noalloc": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_int64, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "rascal_neighbours_static_limit": (C.c_size_t, []),
    "rascal_spherical_expansion": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "rascal_power_spectrum": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "rascal_soap": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                              C.c_void_p, C.c_void_p]),
    "rascal_soap_selected": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_linear_energy": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_gradients": (C.c_int, [C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_radial_exact_fp64": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_set_radial": (C.c_int, [C.c_void_p, C.c_int]),
    "rascal_mlp_num_params": (C.c_int, [C.c_void_p, C.c_int]),
    "rascal_mlp_set_params": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "rascal_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_mlp_targets": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "rascal_mlp_train": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                   C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "rascal_mlp_gradients": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_mlp_eval": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rascal_mlp_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "rascal_mlp_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "rascal_gpr_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_int, C.POINTER(C.c_void_p)]),
    "rascal_gpr_destroy": (None, [C.c_void_p]),
    "rascal_lambda_soap_size": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "rascal_debug_pair_gradients": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "rascal_debug_wait_timeout": (C.c_int, [C.c_void_p, C.c_uint]),
    "rascal_debug_gauss_legendre": (C.c_int, [C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "rascal_debug_real_coupling": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "rascal_lambda_soap": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p]),
    "rascal_gpr_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(System), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
}


def exported_symbols():
    """Names of the entry points the binding declares (all must be exported by the library)."""
    return list(_SIGNATURES)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(status: int):
    if status != RASCAL_OK:
        msg = lib().rascal_last_error()
        raise RascalError(status, msg.decode() if msg else "")
