"""ctypes declarations of the libptycho C-ABI (include/ptycho.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly when the shared library is missing; there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# PTYCHO_LIBRARY=checked loads the checked build (libptycho_checked.so: the
# same entry points with index checks in the kernels)
LIB_PATH = os.path.join(HERE, "libptycho_checked.so" if os.environ.get("PTYCHO_LIBRARY") == "checked"
                        else "libptycho.so")

OK, EINVAL, EOUTOFBOUNDS, ENOMEM, ECUDA, ETIMEDOUT, EBUSY, ENOTFOUND, ECHECK = 0, -1, -2, -3, -4, -5, -6, -7, -8
ECANCELED, ENONFINITE = -9, -10
ERR_NAMES = {EINVAL: "EINVAL", EOUTOFBOUNDS: "EOUTOFBOUNDS", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
             ETIMEDOUT: "ETIMEDOUT", EBUSY: "EBUSY", ENOTFOUND: "ENOTFOUND", ECHECK: "ECHECK",
             ECANCELED: "ECANCELED", ENONFINITE: "ENONFINITE"}


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Geom(C.Structure):
    _fields_ = [("S", C.c_int32), ("K", C.c_int32), ("h", C.c_int32), ("w", C.c_int32),
                ("H", C.c_int32), ("W", C.c_int32), ("dx", C.c_double), ("lam", C.c_double),
                ("dz", C.POINTER(C.c_double)), ("bandlimit", C.c_double), ("loss", C.c_int32),
                ("eps", C.c_double), ("c", C.c_double), ("waves", C.c_int32), ("dft", C.c_int32),
                ("wave_prec", C.c_int32), ("deterministic", C.c_int32)]


class Opt(C.Structure):
    _fields_ = [("lr_O", C.c_float), ("lr_P", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("update_probe", C.c_int32), ("reg_obj_l2", C.c_float),
                ("reg_obj_tikhonov", C.c_float), ("reg_obj_layers", C.c_float), ("reg_probe_l2", C.c_float),
                ("reg_obj_tv", C.c_float), ("reg_obj_layers_tv", C.c_float), ("reg_tv_eps", C.c_float)]


class LsqmlOpt(C.Structure):
    _fields_ = [("beta_O", C.c_float), ("beta_P", C.c_float), ("delta_O", C.c_float), ("delta_P", C.c_float),
                ("gamma", C.c_float)]


class Adam(C.Structure):
    _fields_ = [("mO", C.c_void_p), ("vO", C.c_void_p), ("mP", C.c_void_p), ("vP", C.c_void_p),
                ("t", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("geom", Geom), ("n_pos", C.c_int32), ("pos", C.c_void_p), ("I_exp", C.c_void_p),
                ("O_init", C.c_void_p), ("P_init", C.c_void_p), ("iterations", C.c_int32),
                ("batch", C.c_int32), ("grouping", C.c_int32), ("seed", C.c_uint64), ("opt", Opt)]


class Status(C.Structure):
    _fields_ = [("state", C.c_int32), ("iterations_done", C.c_int32), ("error", C.c_int32),
                ("last_loss", C.c_double), ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("finish_ms", C.c_double)]


class Result(C.Structure):
    _fields_ = [("O", C.c_void_p), ("P", C.c_void_p), ("loss", C.POINTER(C.c_double)), ("n_loss", C.c_int32),
                ("step_ms", C.POINTER(C.c_double)), ("n_step", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("finished", C.c_int64),
                ("failed", C.c_int64), ("queue_depth", C.c_int64), ("admitted_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("launches", C.c_int64), ("positions_per_s", C.c_double),
                ("p50_iter_ms", C.c_double), ("p99_iter_ms", C.c_double)]


P_ = C.c_void_p
I32 = C.c_int32
SIGNATURES = {
    "ptycho_create": (I32, [C.POINTER(Geom), I32, C.c_size_t, C.POINTER(P_)]),
    "ptycho_destroy": (I32, [P_]),
    "ptycho_scratch_bytes": (C.c_size_t, [C.POINTER(Geom), I32, I32]),
    "ptycho_forward": (I32, [P_, P_, P_, P_, I32, P_, P_]),
    "ptycho_adjoint": (I32, [P_, P_, P_, P_, I32, P_, P_, P_, P_, I32, P_]),
    "ptycho_vjp": (I32, [P_, P_, P_, P_, I32, P_, P_, P_, I32, P_]),
    "ptycho_adjoint_positions": (I32, [P_, P_, P_, P_, I32, P_, P_, P_, P_, P_, I32, P_]),
    "ptycho_forward_static": (I32, [C.POINTER(Geom), P_, P_, P_, I32, P_, P_, P_]),
    "ptycho_step": (I32, [P_, P_, P_, C.POINTER(Adam), C.POINTER(Opt), P_, P_, I32, P_, I32, P_, P_]),
    "ptycho_step_host": (I32, [P_, P_, P_, C.POINTER(Adam), C.POINTER(Opt), P_, P_, I32,
                               C.POINTER(C.c_double), C.POINTER(C.c_double), P_]),
    "ptycho_epie_step": (I32, [P_, P_, P_, C.c_float, C.c_float, P_, P_, I32, P_, I32, P_, P_]),
    "ptycho_lsqml_step": (I32, [P_, P_, P_, C.POINTER(LsqmlOpt), P_, P_, P_, P_, P_, P_, I32, P_, I32, P_, P_]),
    "ptycho_exchange_selftest": (I32, [I32]),
    "ptycho_check": (I32, [P_, P_]),
    "ptycho_make_groups": (I32, [I32, I32, C.c_uint64, C.c_int64, I32, P_, P_]),
    "ptycho_set_timing": (I32, [P_, I32]),
    "ptycho_set_step_counter": (I32, [P_, P_]),
    "ptycho_kernel_times": (I32, [P_, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(I32), I32]),
    "ptycho_fft2": (I32, [I32, I32, P_, P_, I32, P_]),
    "ptycho_fft2_dft": (I32, [I32, I32, I32, P_, P_, I32, P_]),
    "ptycho_dft_rows_tc": (I32, [I32, I32, I32, P_, P_, I32, P_]),
    "ptycho_dft_rows_tc_check": (I32, []),
    "ptycho_server_create": (I32, [C.c_size_t, I32, C.POINTER(P_)]),
    "ptycho_server_destroy": (I32, [P_]),
    "ptycho_submit": (I32, [P_, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "ptycho_poll": (I32, [P_, C.c_uint64, C.POINTER(Status), C.POINTER(Result)]),
    "ptycho_wait": (I32, [P_, C.c_uint64, C.c_double]),
    "ptycho_release": (I32, [P_, C.c_uint64]),
    "ptycho_cancel": (I32, [P_, C.c_uint64]),
    "ptycho_server_inject_stall": (I32, [P_, C.c_double]),
    "ptycho_server_stats_get": (I32, [P_, C.POINTER(ServerStats)]),
    "ptycho_fp32_peak_launch": (I32, [I32, I32, P_, C.POINTER(C.c_double), P_]),
    "ptycho_fp32_peak_sink_elems": (I32, []),
    "ptycho_kernels_launched": (C.c_uint64, []),
    "ptycho_last_error": (C.c_char_p, []),
    "ptycho_version": (C.c_char_p, []),
    "ptycho_build_checked": (C.c_int32, []),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2505_14372_b300.build` (there is no fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> int:
    if rc != OK:
        raise PtychoError(rc, lib().ptycho_last_error().decode(errors="replace"))
    return rc
