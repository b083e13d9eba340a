"""ctypes declarations of include/sdmm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

SDMM_ETAB_FLOATS = 36
SDMM_QTAB_FLOATS = 36
SDMM_MAX_K = 32

STATUS = {0: "SDMM_OK", 1: "SDMM_ERR_INVALID_ARG", 2: "SDMM_ERR_CUDA", 4: "SDMM_ERR_UNSUPPORTED",
          5: "SDMM_ERR_WORKSPACE"}

# exported symbols (kept in sync with include/sdmm.h; a test checks both)
SYMBOLS = ["sdmm_config_default", "sdmm_last_error", "sdmm_version", "sdmm_fit_workspace_size",
           "sdmm_init_regions", "sdmm_fit_regions", "sdmm_prepare", "sdmm_condition",
           "sdmm_sample", "sdmm_pdf", "sdmm_objective", "sdmm_objective_backward",
           "sdmm_fit_plan_create", "sdmm_fit_plan_run", "sdmm_fit_plan_enable_timing",
           "sdmm_fit_plan_staging_size", "sdmm_fit_plan_run_host",
           "sdmm_fit_plan_timing", "sdmm_fit_plan_destroy", "sdmm_autotune",
           "sdmm_fit_regions_noalloc", "sdmm_tc_selftest", "sdmm_wait_selftest", "sdmm_validate_samples", "sdmm_kdtree_grid", "sdmm_kdtree_lookup",
           "sdmm_kdtree_workspace_size", "sdmm_kdtree_bin", "sdmm_kdtree_refine", "sdmm_gather_regions",
           "sdmm_product_sample", "sdmm_product_pdf", "sdmm_query_workspace_size", "sdmm_sample_binned",
           "sdmm_pdf_binned"]

SDMM_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


class Config(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("min_samples", ctypes.c_int32),
                ("eta_mode", ctypes.c_int32), ("estep_density", ctypes.c_int32),
                ("prior_scale_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("cov_update", ctypes.c_int32), ("dir_coords", ctypes.c_int32),
                ("eta_alpha", ctypes.c_double), ("eta_beta", ctypes.c_double),
                ("prior_q", ctypes.c_double), ("prior_a", ctypes.c_double),
                ("prior_B_pos", ctypes.c_double), ("prior_B_dir", ctypes.c_double)]


class State(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("pi", "mu_x", "mu_w", "L", "S0", "S2", "Wbar", "n_seen", "step_j", "status",
                 "etab", "qtab")]


class Samples(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("px", "py", "pz", "ox", "oy", "oz", "w", "offsets")] + \
               [("R", ctypes.c_int64), ("N", ctypes.c_int64)]


class KdTree(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_void_p), ("split", ctypes.c_void_p), ("left", ctypes.c_void_p),
                ("leaf", ctypes.c_void_p), ("n_nodes", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("cap_nodes", ctypes.c_int32), ("cap_leaves", ctypes.c_int32)]


class SampleBuffers(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("px", "py", "pz", "ox", "oy", "oz", "w", "offsets")] + \
               [("R", ctypes.c_int64), ("N", ctypes.c_int64)]


class BsdfLobes(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("L", ctypes.c_void_p), ("J", ctypes.c_int32)]


class Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("dims", ctypes.c_int32 * 3)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PC = ctypes.POINTER(Config)
_PS = ctypes.POINTER(State)
_PSm = ctypes.POINTER(Samples)
_PG = ctypes.POINTER(Grid)


def _declare(L):
    L.sdmm_config_default.restype = None
    L.sdmm_config_default.argtypes = [_PC, _I32]
    L.sdmm_last_error.restype = ctypes.c_char_p
    L.sdmm_last_error.argtypes = []
    L.sdmm_version.restype = ctypes.c_char_p
    L.sdmm_version.argtypes = []
    sig = {
        "sdmm_fit_workspace_size": [_PC, _I64, _I64, ctypes.POINTER(ctypes.c_size_t)],
        "sdmm_init_regions": [_PC, _PSm, _P, _P, _PS, _P],
        "sdmm_fit_regions": [_PC, _PSm, _I32, _P, _PS, _P, _P, ctypes.c_size_t, _P],
        "sdmm_prepare": [_PC, _I64, _PS, _P, _P, _P],
        "sdmm_condition": [_PC, _PS, _I64, _I64, _P, _P, _PG, _P, _P, _P, _P],
        "sdmm_sample": [_PC, _PS, _I64, _I64, _P, _P, _PG, ctypes.c_uint64, _P, _P, _P, _P, _P],
        "sdmm_pdf": [_PC, _PS, _I64, _I64, _P, _P, _PG, _P, _P, _P],
        "sdmm_objective": [_PC, _PSm, _P, _PS, _P, _P, ctypes.c_size_t, _P],
        "sdmm_objective_backward": [_PC, _PSm, _P, _PS, _P, _P, _P, _P, _P, ctypes.c_size_t, _P],
        "sdmm_fit_plan_create": [_PC, _I64, _I64, _I32, _PS, _P, ctypes.c_size_t, _P,
                                 ctypes.POINTER(ctypes.c_void_p)],
        "sdmm_fit_plan_run": [_P, _PSm, _P, _P, _P],
        "sdmm_fit_plan_staging_size": [_P, ctypes.POINTER(ctypes.c_size_t)],
        "sdmm_fit_plan_run_host": [_P, _PSm, _P, ctypes.c_size_t, _P, _P, _P],
        "sdmm_fit_plan_enable_timing": [_P, _I32],
        "sdmm_fit_plan_timing": [_P, _P, _I32, ctypes.POINTER(_I32)],
        "sdmm_fit_plan_destroy": [_P],
        "sdmm_autotune": [_PC, _PSm, _PS, _P, ctypes.c_size_t, _P, ctypes.POINTER(_I32),
                          ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)],
        "sdmm_fit_regions_noalloc": [_PC, _PSm, _I32, _P, _PS, _P, _P],
        "sdmm_tc_selftest": [_I32, _I32, _I32, _P, _P, _P, _I32, _P, _P],
        "sdmm_wait_selftest": [ctypes.c_int64, _I32, _P, _P, _P],
        "sdmm_validate_samples": [_PSm, ctypes.c_float, _P, _P],
        "sdmm_kdtree_grid": [ctypes.POINTER(KdTree), _I32, _P],
        "sdmm_kdtree_lookup": [ctypes.POINTER(KdTree), _I64, _P, _P, _P, _P, _P],
        "sdmm_kdtree_workspace_size": [ctypes.POINTER(KdTree), _I64, ctypes.POINTER(ctypes.c_size_t)],
        "sdmm_kdtree_bin": [ctypes.POINTER(KdTree), _PSm, ctypes.POINTER(SampleBuffers), _P, ctypes.c_size_t, _P],
        "sdmm_kdtree_refine": [ctypes.POINTER(KdTree), _I64, _PSm, ctypes.POINTER(SampleBuffers), _P, _P,
                               ctypes.c_size_t, _P],
        "sdmm_gather_regions": [_I32, _I64, _P, _PS, _PS, _P],
        "sdmm_product_sample": [_PC, _PS, _I64, _I64, _P, _P, _PG, ctypes.POINTER(BsdfLobes), ctypes.c_uint64, _P,
                                _P, _P, _P, _P],
        "sdmm_product_pdf": [_PC, _PS, _I64, _I64, _P, _P, _PG, ctypes.POINTER(BsdfLobes), _P, _P, _P],
        "sdmm_query_workspace_size": [_I64, _I64, ctypes.POINTER(ctypes.c_size_t)],
        "sdmm_sample_binned": [_PC, _PS, _I64, _I64, _P, _P, _PG, ctypes.c_uint64, _P, _P, _P, _P, _P,
                               ctypes.c_size_t, _P],
        "sdmm_pdf_binned": [_PC, _PS, _I64, _I64, _P, _P, _PG, _P, _P, _P, ctypes.c_size_t, _P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.restype = _I
        f.argtypes = args


def load(build_if_missing: bool = True):
    """Loads libsdmm.so (building it with nvcc first if it is missing).

    There is no fallback: if the library cannot be built or loaded, this
    raises."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB) or not _build.up_to_date():
                if not build_if_missing:
                    raise RuntimeError(f"{_build.LIB} is missing; run paper_2111_13094_gb300.build")
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            _declare(L)
            _lib = L
    return _lib


class SdmmError(RuntimeError):
    pass


def check(code: int, what: str = ""):
    if code != 0:
        msg = load().sdmm_last_error().decode(errors="replace")
        raise SdmmError(f"{what}: {STATUS.get(code, code)}: {msg}")
