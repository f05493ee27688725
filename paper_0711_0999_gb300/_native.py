"""ctypes declarations of the C ABI in ``include/nedmft.h`` (argument marshalling only).

The shared library is loaded on first use.  There is no fallback: if
``libnedmft.so`` is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnedmft.so")

c_double = ctypes.c_double
c_int32 = ctypes.c_int32
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p

NEDMFT_OK = 0
NEDMFT_EINVAL = -1
NEDMFT_ENOMEM = -2
NEDMFT_ECUDA = -3
NEDMFT_ESINGULAR = -4
NEDMFT_ETIMEOUT = -5
NEDMFT_ENOTCONV = 1

FP64 = 0
MIXED_BF16 = 1
PRECISIONS = {"fp64": FP64, "mixed_bf16": MIXED_BF16}


class Contour(ctypes.Structure):
    _fields_ = [("t_min", c_double), ("t_max", c_double), ("dt", c_double), ("beta", c_double),
                ("dtau", c_double), ("n_t", c_int32), ("n_tau", c_int32), ("n_c", c_int32)]


class Model(ctypes.Structure):
    _fields_ = [("U", c_double), ("E", c_double), ("w1", c_double), ("mu", c_double)]


class NedmftError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"nedmft error {code}: {message}")
        self.code = code


PC = ctypes.POINTER(Contour)
PM = ctypes.POINTER(Model)
PD = ctypes.POINTER(c_double)
PI = ctypes.POINTER(c_int32)

# name -> (restype, argtypes); every symbol declared in include/nedmft.h
SIGNATURES = {
    "nedmft_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nedmft_last_error": (ctypes.c_char_p, []),
    "nedmft_version": (ctypes.c_char_p, []),
    "nedmft_check_status": (ctypes.c_int, [c_void_p]),
    "nedmft_set_wait_limit": (ctypes.c_int, [c_double, c_void_p]),
    "nedmft_wait_selftest": (ctypes.c_int, [c_void_p]),
    "nedmft_instrument": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "nedmft_instrument_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), PD, PD,
                                               PD]),
    "nedmft_contour_grid": (ctypes.c_int, [c_double, c_double, c_double, c_double, c_double, PC, c_void_p, c_void_p]),
    "nedmft_gauss_hermite": (ctypes.c_int, [c_int32, PD, PD]),
    "nedmft_quadrature_grid": (ctypes.c_int, [c_int32, PD, PD, PD]),
    "nedmft_quadrature_grid_avg": (ctypes.c_int, [c_int32, PD, PD, PD]),
    "nedmft_extrapolate_current": (ctypes.c_int, [c_int32, PD, PD, PI, ctypes.POINTER(c_void_p), c_void_p, c_int32,
                                                  c_void_p, c_void_p, c_void_p]),
    "nedmft_moments": (ctypes.c_int, [PC, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nedmft_dos": (ctypes.c_int, [PC, c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p]),
    "nedmft_g0_build": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "nedmft_lattice_workspace_size": (c_size_t, [PC, c_int32, ctypes.c_int, c_int32]),
    "nedmft_lattice_gloc": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_int,
                                           c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nedmft_current": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_int,
                                      c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nedmft_lattice_gloc_static": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                                  c_void_p, c_void_p, c_void_p, c_void_p]),
    "nedmft_impurity_workspace_size": (c_size_t, [PC]),
    "nedmft_impurity_update": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                              c_void_p]),
    "nedmft_mlp_param_count": (c_int32, []),
    "nedmft_mlp_workspace_size": (c_size_t, [c_int32]),
    "nedmft_mlp_forward": (ctypes.c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nedmft_mlp_grad": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_size_t,
                                       c_void_p]),
    "nedmft_mlp_adam": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float, c_void_p]),
    "nedmft_mlp_features": (ctypes.c_int, [PC, PM, c_void_p, c_void_p]),
    "nedmft_mlp_target": (ctypes.c_int, [PC, PM, c_void_p, c_double, c_void_p, c_void_p]),
    "nedmft_mlp_sample": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_int64, c_int32, ctypes.c_uint64, ctypes.c_int64,
                                         c_void_p, c_void_p, c_void_p]),
    "nedmft_sigma_warm_start_workspace_size": (c_size_t, [PC]),
    "nedmft_sigma_warm_start": (ctypes.c_int, [PC, PM, c_void_p, c_int32, PD, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nedmft_lattice_autotune": (ctypes.c_int, [PC, PM, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_int,
                                               PI, c_int32, PI, PD, c_void_p, c_size_t, c_void_p]),
    "nedmft_lattice_batch": (c_int32, [PC, c_int32, ctypes.c_int]),
    "nedmft_lattice_block_width": (c_int32, [PC, c_int32, ctypes.c_int]),
    "nedmft_lattice_set_tuning": (ctypes.c_int, [PC, c_int32, ctypes.c_int, c_int32, c_int32]),
    "nedmft_dmft_batch_workspace_size": (c_size_t, [c_int32, PC, c_int32, ctypes.c_int]),
    "nedmft_dmft_solve_batch": (ctypes.c_int, [c_int32, PC, PM, c_int32, ctypes.c_int, ctypes.POINTER(c_void_p),
                                               c_double, c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                               ctypes.POINTER(c_void_p), PI, PD, PI, c_void_p, c_size_t, c_void_p]),
    "nedmft_dmft_workspace_size": (c_size_t, [PC, c_int32, ctypes.c_int]),
    "nedmft_dmft_solve": (ctypes.c_int, [PC, PM, c_int32, ctypes.c_int, c_void_p, c_double, c_int32, c_void_p,
                                         c_void_p, c_void_p, PI, PD, c_void_p, c_size_t, c_void_p]),
}

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise NedmftError(NEDMFT_ECUDA, f"{LIB_PATH} is missing: build it with "
                                      "`python -c 'import __graft_entry__ as g; g.build()'`")
                handle = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
                for name, (res, args) in SIGNATURES.items():
                    fn = getattr(handle, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = handle
    return _lib


def check(rc: int, allow_warning: bool = False) -> int:
    if rc == NEDMFT_OK or (allow_warning and rc > 0):
        return rc
    msg = lib().nedmft_last_error().decode() or lib().nedmft_status_string(rc).decode()
    raise NedmftError(rc, msg)
