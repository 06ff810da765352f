"""ctypes binding of include/swe_exprb.h (argument marshalling only).

Every computation runs in the CUDA library; this module converts torch CUDA
float64 tensors to device pointers, Python lists to host arrays and status
codes to exceptions.  Loading fails loudly when the library has not been
built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SWE_OK = 0
SWE_ERR_INVALID_ARG, SWE_ERR_NOMEM, SWE_ERR_NOCONV, SWE_ERR_NONFINITE, SWE_ERR_TIMEOUT, SWE_ERR_CUDA = -1, -2, -3, -4, -5, -6
ERRORS = {-1: "INVALID_ARG", -2: "NOMEM", -3: "NOCONV", -4: "NONFINITE", -5: "TIMEOUT", -6: "CUDA"}
SCHEMES = {"epi2": 0, "exprb42": 1, "pexprb43": 2, "exprb53": 3, "epi3": 4}

EXPORTS = ["swe_phi_opts_default", "swe_create_grid", "swe_create_grid_host", "swe_grid_export",
           "swe_destroy_grid", "swe_grid_query",
           "swe_grid_cell_centres", "swe_grid_cell_areas", "swe_rhs", "swe_jv", "swe_jv_noalloc",
           "swe_jtv", "swe_dqtv", "swe_diagnostics", "swe_grid_set_topography", "phi_action",
           "swe_scheme_state_create", "swe_scheme_state_reset", "swe_scheme_state_destroy",
           "exprb_step", "exprb_step_adjoint", "swe_profile_enable", "swe_profile_read", "swe_device_status",
           "swe_last_error", "swe_ensemble_create", "swe_ensemble_destroy", "swe_ensemble_set_state",
           "swe_ensemble_get_state", "swe_ensemble_run", "swe_ensemble_reset", "swe_ensemble_tune",
           "swe_ensemble_stats", "swe_ensemble_shape", "swe_ensemble_work", "swe_selftest_wait"]


class PhiOptsC(C.Structure):
    _fields_ = [("tol", C.c_double), ("tol_mode", C.c_int), ("m_init", C.c_int),
                ("m_max", C.c_int), ("iom", C.c_int), ("delta", C.c_double),
                ("gamma", C.c_double), ("kappa", C.c_double), ("max_reject", C.c_int),
                ("m_carry", C.c_int), ("replay", C.POINTER(C.c_double)), ("n_replay", C.c_int),
                ("precision", C.c_int), ("max_substeps", C.c_int)]


class PhiAttemptC(C.Structure):
    _fields_ = [("t", C.c_double), ("tau", C.c_double), ("omega", C.c_double),
                ("m", C.c_int), ("accepted", C.c_int), ("call", C.c_int), ("pad", C.c_int)]


class PhiStatsC(C.Structure):
    _fields_ = [("n_jv", C.c_int), ("n_substeps", C.c_int), ("n_reject", C.c_int),
                ("m_last", C.c_int), ("m_max_used", C.c_int), ("status", C.c_int),
                ("trace", C.POINTER(PhiAttemptC)), ("trace_cap", C.c_int), ("n_trace", C.c_int)]


class ProfileC(C.Structure):
    _fields_ = [("phi_ms", C.c_double), ("call_ms", C.c_double), ("phi_flop", C.c_double),
                ("phi_bytes", C.c_double), ("phi_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("iom2_iterations", C.c_int64), ("w_jv", C.c_int64), ("comb_terms", C.c_int64),
                ("phase_ms", C.c_double * 10), ("phi_table_bytes", C.c_double)]


class SweError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None) -> C.CDLL:
    """Load libswe_exprb.so (built by build.build()); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    L.swe_phi_opts_default.argtypes = [C.POINTER(PhiOptsC)]
    L.swe_phi_opts_default.restype = None
    L.swe_create_grid.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                  C.POINTER(vp)]
    L.swe_create_grid_host.argtypes = L.swe_create_grid.argtypes
    L.swe_grid_export.argtypes = [vp, C.c_char_p, vp, C.c_int64]
    L.swe_destroy_grid.argtypes = [vp]
    L.swe_destroy_grid.restype = None
    L.swe_grid_query.argtypes = [vp, i64p, i64p, i64p, dp]
    L.swe_grid_cell_centres.argtypes = [vp, dp]
    L.swe_grid_cell_areas.argtypes = [vp, dp]
    L.swe_rhs.argtypes = [vp, vp, vp, vp]
    L.swe_jv.argtypes = [vp, vp, vp, vp, vp]
    L.swe_jv_noalloc.argtypes = [vp, vp, vp, vp, vp]
    L.swe_jtv.argtypes = [vp, vp, vp, vp, vp]
    L.swe_diagnostics.argtypes = [vp, vp, dp, vp]
    L.swe_grid_set_topography.argtypes = [vp, dp]
    L.swe_dqtv.argtypes = [vp, vp, vp, vp, vp]
    L.phi_action.argtypes = [vp, vp, C.c_double, C.c_int, C.POINTER(vp), C.c_int, dp, C.POINTER(vp),
                             C.POINTER(PhiOptsC), C.POINTER(PhiStatsC), vp]
    L.swe_scheme_state_create.argtypes = [vp, C.POINTER(vp)]
    L.swe_scheme_state_reset.argtypes = [vp]
    L.swe_scheme_state_destroy.argtypes = [vp]
    L.swe_scheme_state_destroy.restype = None
    L.exprb_step.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, C.POINTER(PhiOptsC),
                             C.POINTER(PhiStatsC), vp]
    L.exprb_step_adjoint.argtypes = [vp, C.c_int, C.c_double, vp, C.POINTER(PhiAttemptC), C.c_int, vp, vp,
                                     C.POINTER(PhiOptsC), C.POINTER(PhiStatsC), vp]
    L.swe_profile_enable.argtypes = [vp, C.c_int]
    L.swe_profile_read.argtypes = [vp, C.POINTER(ProfileC), vp]
    L.swe_device_status.argtypes = [vp, vp]
    L.swe_selftest_wait.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_int), vp]
    L.swe_ensemble_create.argtypes = [C.POINTER(vp), C.c_int, dp, C.POINTER(C.c_int),
                                      C.POINTER(PhiOptsC), C.POINTER(vp)]
    L.swe_ensemble_destroy.argtypes = [vp]
    L.swe_ensemble_destroy.restype = None
    L.swe_ensemble_set_state.argtypes = [vp, C.c_int, vp, vp]
    L.swe_ensemble_get_state.argtypes = [vp, C.c_int, vp, vp]
    L.swe_ensemble_run.argtypes = [vp, vp]
    L.swe_ensemble_reset.argtypes = [vp, vp]
    L.swe_ensemble_tune.argtypes = [vp, C.c_int, vp]
    L.swe_ensemble_stats.argtypes = [vp, C.POINTER(PhiStatsC), dp, C.POINTER(C.c_int), vp]
    ip = C.POINTER(C.c_int)
    L.swe_ensemble_shape.argtypes = [vp, ip, ip, ip, ip, ip]
    L.swe_ensemble_work.argtypes = [vp, dp, vp]
    L.swe_last_error.argtypes = []
    L.swe_last_error.restype = C.c_char_p
    for name in ("swe_create_grid", "swe_create_grid_host", "swe_grid_export", "swe_grid_query", "swe_grid_cell_centres", "swe_grid_cell_areas",
                 "swe_rhs", "swe_jv", "swe_jv_noalloc", "swe_jtv", "swe_dqtv", "swe_diagnostics", "swe_grid_set_topography", "phi_action",
                 "swe_scheme_state_create",
                 "swe_scheme_state_reset", "exprb_step", "exprb_step_adjoint", "swe_device_status", "swe_profile_enable",
                 "swe_profile_read", "swe_ensemble_create", "swe_ensemble_set_state",
                 "swe_ensemble_get_state", "swe_ensemble_run", "swe_ensemble_reset", "swe_ensemble_tune",
                 "swe_ensemble_stats", "swe_ensemble_shape", "swe_ensemble_work", "swe_selftest_wait"):
        getattr(L, name).restype = C.c_int
    _LIB = L
    return L


def check(rc: int) -> None:
    if rc != SWE_OK:
        raise SweError(rc, load().swe_last_error().decode())


def default_opts(**kw) -> PhiOptsC:
    o = PhiOptsC()
    load().swe_phi_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "replay":
            continue
        setattr(o, k, v)
    return o
