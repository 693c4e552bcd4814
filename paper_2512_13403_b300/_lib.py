"""ctypes binding of libdh.so (include/dh.h): argument marshalling only.

Every function keeps the C name and signature; all numerical work happens in the CUDA library.
Loading fails loudly if the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdh.so")

DH_OK, DH_ERR_ARG, DH_ERR_CUDA, DH_ERR_NONFINITE, DH_ERR_POSITIVITY, DH_ERR_MG_NOCONV, DH_ERR_STATE = range(7)
DH_F32, DH_F64 = 0, 1
KERNEL_KINDS = {"stage1": 0, "stage2": 1, "prologue": 2, "reduce": 3, "sources": 4, "mg": 5,
                "adjoint": 6, "conv": 7}


class DhConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("precision", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("gamma", C.c_double), ("cfl", C.c_double), ("dt_max", C.c_double),
        ("forcing", C.c_int), ("ou_tau", C.c_double), ("ou_arms", C.c_double),
        ("ou_seed", C.c_ulonglong),
        ("cooling", C.c_int), ("t_floor", C.c_double), ("cool_frac", C.c_double),
        ("nsub_max", C.c_int),
        ("gravity", C.c_int), ("four_pi_G", C.c_double), ("mg_tol", C.c_double),
        ("mg_max_cycles", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int),
        ("mg_smoother", C.c_int), ("mg_omega", C.c_double), ("mg_cycle", C.c_int),
        ("limiter", C.c_int), ("integrator", C.c_int),
        ("c_cool", C.c_double),
    ]


class DhMetrics(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("dt", C.c_double), ("nstep", C.c_longlong), ("flags", C.c_uint),
        ("cool_max_substeps", C.c_int), ("slope_fallbacks", C.c_longlong),
        ("mg_cycles", C.c_int), ("mg_residual", C.c_double),
        ("totals", C.c_double * 5), ("rho_min", C.c_double), ("p_min", C.c_double),
    ]


DH_FLAG_NONFINITE, DH_FLAG_POSITIVITY, DH_FLAG_MG_NOCONV, DH_FLAG_COOL_CAP = 1, 2, 4, 8

_P = C.c_void_p
_SIGNATURES = {
    "dh_config_default": (None, [C.POINTER(DhConfig), C.c_int, C.c_int, C.c_int]),
    "dh_create": (C.c_int, [C.POINTER(DhConfig), _P, C.POINTER(_P)]),
    "dh_destroy": (None, [_P]),
    "dh_init_state": (C.c_int, [_P, _P, C.c_int]),
    "dh_get_state": (C.c_int, [_P, _P, C.c_int]),
    "dh_step": (C.c_int, [_P, C.c_double, C.POINTER(C.c_double)]),
    "dh_advance": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "dh_get_time": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "dh_compute_dt": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "dh_get_metrics": (C.c_int, [_P, C.POINTER(DhMetrics)]),
    "dh_conserved_totals": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "dh_forcing_field": (C.c_int, [_P, _P, C.c_int]),
    "dh_forcing_modes": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "dh_set_forcing_modes": (C.c_int, [_P, C.POINTER(C.c_double), C.c_int]),
    "dh_downsample": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "dh_get_potential": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "dh_solve_poisson": (C.c_int, [_P, _P, C.c_int]),
    "dh_reset_potential": (C.c_int, [_P]),
    "dh_fft_poisson": (C.c_int, [_P, _P, C.c_int, _P, C.c_int]),
    "dh_adjoint_advance": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int]),
    "dh_adjoint_advance_dt": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, _P, _P, C.c_int]),
    "dh_conserved_totals_static": (C.c_int, [_P, C.c_int, C.c_longlong, _P, _P]),
    "dh_save": (C.c_int, [_P, C.c_char_p]),
    "dh_load": (C.c_int, [_P, C.c_char_p]),
    "dh_conv_padded_rows": (C.c_longlong, [C.c_int, C.c_int, C.c_int]),
    "dh_conv_pad": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "dh_conv_unpad": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "dh_pack_conv_weights": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "dh_conv3d_bf16": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int, _P, _P, _P, C.c_int,
                                 C.c_int, C.c_int, C.c_int, _P, _P]),
    "dh_conv3d_wgrad_bf16": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_int, _P, C.c_int, _P, _P, _P]),
    "dh_cnn_param_count": (C.c_longlong, []),
    "dh_cnn_create": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, C.POINTER(_P)]),
    "dh_cnn_param_count_form": (C.c_longlong, [C.c_int]),
    "dh_cnn_create_form": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(_P)]),
    "dh_cnn_vjp": (C.c_int, [_P, _P, _P, _P]),
    "dh_cnn_destroy": (None, [_P]),
    "dh_cnn_set_params": (C.c_int, [_P, _P, C.POINTER(C.c_float)]),
    "dh_cnn_forward": (C.c_int, [_P, _P, _P]),
    "dh_cnn_backward": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double)]),
    "dh_cnn_correct_state": (C.c_int, [_P, _P, C.c_double, C.c_double, C.c_double]),
    "dh_cnn_rollout_misfit": (C.c_int, [_P, _P, _P, C.POINTER(C.c_float), C.c_double, _P, C.c_int, _P]),
    "dh_cnn_floor_vjp": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.c_double]),
    "dh_cnn_field_moments": (C.c_int, [_P, _P, _P, C.c_longlong, C.POINTER(C.c_double)]),
    "dh_axpy": (C.c_int, [C.c_longlong, C.c_double, _P, _P, _P]),
    "dh_adam_step": (C.c_int, [_P, _P, _P, _P, C.c_longlong, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_int, _P]),
    "dh_set_corrector": (C.c_int, [_P, _P, C.POINTER(C.c_float)]),
    "dh_set_corrector_form": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_float)]),
    "dh_correct": (C.c_int, [_P]),
    "dh_set_correct_every_step": (C.c_int, [_P, C.c_int]),
    "dh_profile_enable": (C.c_int, [_P, C.c_int]),
    "dh_profile_read": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double)]),
    "dh_launch_count": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "dh_last_error": (C.c_char_p, [_P]),
    "dh_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def exported_names():
    return list(_SIGNATURES)


def load(path: str = LIB_PATH):
    """Loads libdh.so (raises if it is absent) and declares every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DhError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


def status_name(s: int) -> str:
    return load().dh_status_string(s).decode()


def check(status: int, ctx=None):
    if status != DH_OK:
        msg = load().dh_last_error(ctx).decode(errors="replace")
        raise DhError(status, msg)
