"""ctypes declarations of the C-ABI in include/mp_poisson.h.

Loading fails loudly (ImportError) when the compiled library is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MP_OK = 0
MP_ERR_INVALID_ARG = 1
MP_ERR_NOT_CONVERGED = 2
MP_ERR_DIVERGED = 3
MP_ERR_CUDA = 4
MP_ERR_OOM = 5
MP_ERR_TIMEOUT = 6
MP_ERR_NO_NET = 7

MP_NOALLOC_MAX_CELLS = 134217728

MP_BC_PERIODIC = 0
MP_BC_NEUMANN = 1
MP_BC_DIRICHLET = 2
MP_BC_NEUMANN_DIRICHLET = 3
MP_BC_DIRICHLET_NEUMANN = 4


class mp_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class mp_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("method", ctypes.c_int),
        ("initial_guess", ctypes.c_int),
        ("max_iters", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("nu_growth", ctypes.c_int),
        ("nu_max", ctypes.c_int),
        ("inner_rtol", ctypes.c_double),
        ("inner_max", ctypes.c_int),
        ("net_check", ctypes.c_int),
        ("deflate", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("label_limit", ctypes.c_int),
        ("coarse_cluster", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class mp_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("outer_steps", ctypes.c_int),
        ("relres", ctypes.c_double),
        ("r0", ctypes.c_double),
        ("used_net", ctypes.c_int),
        ("net_relres", ctypes.c_double),
        ("levels", ctypes.c_int),
        ("coarse_n", ctypes.c_int),
        ("components", ctypes.c_int),
    ]


class mp_kernel_prof(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 40),
        ("level", ctypes.c_int),
        ("cells", ctypes.c_longlong),
        ("launches", ctypes.c_longlong),
        ("total_ms", ctypes.c_double),
        ("alg_bytes", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "mp_opts_default": (None, [ctypes.POINTER(mp_opts)]),
    "mp_status_str": (ctypes.c_char_p, [_I]),
    "mp_poisson_setup": (_I, [ctypes.POINTER(_P), mp_grid, _D, _IP, _P, _D, _D, _D,
                              ctypes.POINTER(mp_opts)]),
    "mp_poisson_set_geometry": (_I, [_P, _P, _D, _D, _D]),
    "mp_poisson_set_mass_flux": (_I, [_P, _P]),
    "mp_poisson_deflated_energy": (_I, [_P, _P, _P, _P, _DP]),
    "mp_poisson_set_opts": (_I, [_P, ctypes.POINTER(mp_opts)]),
    "mp_poisson_solve": (_I, [_P, _P, _P, _D, _IP, _DP, _I, _IP]),
    "mp_poisson_project_step": (_I, [_P, _P, _P, _P, _P, _D, _IP]),
    "mp_poisson_project_step_host": (_I, [_P, _P, _P, _P, _P, _D, _IP]),
    "mp_poisson_apply": (_I, [_P, _P, _P]),
    "mp_poisson_divergence": (_I, [_P, _P, _P, _P, _P]),
    "mp_poisson_rhs": (_I, [_P, _P, _P]),
    "mp_poisson_project": (_I, [_P, _P, _P, _P, _P]),
    "mp_poisson_get_fields": (_I, [_P, _P, _P, _P, _P, _P]),
    "mp_poisson_get_stats": (_I, [_P, ctypes.POINTER(mp_stats)]),
    "mp_poisson_set_profiling": (_I, [_P, _I]),
    "mp_poisson_get_profile": (_I, [_P, ctypes.POINTER(mp_kernel_prof), _I, _IP]),
    "mp_poisson_rhs_noalloc": (_I, [ctypes.c_longlong, _P, _P, _P, _P]),
    "mp_poisson_destroy": (None, [_P]),
    "mp_poisson_set_net": (_I, [_P, _P]),
    "mp_poisson_get_components": (_I, [_P, _P, _IP]),
    "mp_conv3d_fwd": (_I, [_I, _I, _I, _P, _I, _I, _P, _I, _P, _P, _I, _I, _P, _P, _P]),
    "mp_conv3d_wgrad": (_I, [_I, _I, _I, _P, _I, _I, _P, _I, _P, _I, _P, _P]),
    "mp_net_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _P]),
    "mp_net_dims": (_I, [_P, _IP, _IP, _IP]),
    "mp_net_param_count": (ctypes.c_size_t, [_P]),
    "mp_net_launches": (ctypes.c_ulonglong, [_P]),
    "mp_net_set_params": (_I, [_P, _P]),
    "mp_net_train_step_grad": (_I, [_P, _P, ctypes.c_float, _I]),
    "mp_net_get_adam": (_I, [_P, _P, _P]),
    "mp_net_set_adam": (_I, [_P, _P, _P]),
    "mp_net_get_params": (_I, [_P, _P]),
    "mp_net_features": (_I, [_P, _P, _P, _D, _D, _DP]),
    "mp_net_get_input2": (_I, [_P, _P]),
    "mp_net_set_input2": (_I, [_P, _P]),
    "mp_net_forward": (_I, [_P, _P]),
    "mp_net_train_step": (_I, [_P, _P, ctypes.c_float, _I, _DP]),
    "mp_net_loss_grad": (_I, [_P, _P, _P, _DP]),
    "mp_net_test_wait_timeout": (_I, [_I]),
    "mp_net_set_input": (_I, [_P, _P]),
    "mp_net_backward": (_I, [_P, _P, _P]),
    "mp_net_pressure": (_I, [_P, _D, _P]),
    "mp_net_set_stream": (_I, [_P, _P]),
    "mp_net_set_loss": (_I, [_P, _I, _D, _D, _IP]),
    "mp_net_features_at": (_I, [_P, _I, _P, _P, _D, _D, _DP]),
    "mp_net_pressure_at": (_I, [_P, _I, _IP, _D, _P]),
    "mp_net_make_target": (_I, [_P, _P, _P]),
    "mp_net_destroy": (None, [_P]),
}

_lib = None


def path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(
            "mp_poisson CUDA library not built (%s); run __graft_entry__.build() or "
            "python -m paper_2312_11740_gb300.build" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
