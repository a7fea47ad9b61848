"""ctypes binding of libdeblur.so (declarations in include/deblur.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. Loading fails loudly when the shared library is missing; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdeblur.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "deblur.h")

SOLVERS = {"irls": 0, "mm": 1, "sb": 2}
WAVELETS = {"haar": 0, "db4": 1}
TRANSFERS = {"I": 0, "X": 1, "D": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}
STATUS = {0: "DB_OK", 1: "DB_EINVAL", 2: "DB_ENOMEM", 3: "DB_ECUDA", 4: "DB_ETIMEOUT",
          5: "DB_EBUSY", 6: "DB_ECANCELLED"}


class DbOpts(C.Structure):
    _fields_ = [("tol_fine", C.c_double), ("tol_coarse", C.c_double), ("kmax", C.c_int),
                ("eps_irls", C.c_double), ("eps_mm", C.c_double), ("tau_sb", C.c_double),
                ("lsqr_atol", C.c_double), ("lsqr_btol", C.c_double), ("lsqr_conlim", C.c_double),
                ("lsqr_maxit", C.c_int), ("lsqr_warm_start", C.c_int), ("precision", C.c_int),
                ("barrier_timeout_us", C.c_int), ("fine_direct", C.c_int)]


class DbGcvOpts(C.Structure):
    _fields_ = [("grid_points", C.c_int), ("log10_gamma_lo", C.c_double), ("log10_gamma_hi", C.c_double),
                ("refine_tol_log10", C.c_double), ("gcv_estimates", C.c_int), ("proj_dim", C.c_int),
                ("proj_dim_max", C.c_int), ("gamma_fixed", C.c_double), ("exact_max_pixels", C.c_int)]


class DbStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("lsqr_launches", C.c_uint64), ("lsqr_ms", C.c_double),
                ("lsqr_pixel_iters_irls", C.c_double), ("lsqr_pixel_iters_other", C.c_double),
                ("gcv_calls", C.c_uint64), ("outer_iterations", C.c_uint64), ("gcv_ms", C.c_double),
                ("lsqr_fine_launches", C.c_uint64), ("lsqr_fine_ms", C.c_double),
                ("lsqr_fine_pixel_iters_irls", C.c_double), ("lsqr_fine_pixel_iters_other", C.c_double),
                ("lsqr_direct_solves", C.c_uint64), ("blur_direct_launches", C.c_uint64)]


class DbRequest(C.Structure):
    _fields_ = [("b", C.c_void_p), ("m", C.c_int), ("psf", C.c_void_p), ("psf_size", C.c_int),
                ("solver", C.c_int), ("wavelet", C.c_int), ("levels", C.c_int), ("transfer", C.c_int),
                ("x", C.c_void_p), ("mu_per_level", C.c_void_p), ("iters_per_level", C.c_void_p),
                ("inner_iters_per_level", C.c_void_p)]


class DbServerOpts(C.Structure):
    _fields_ = [("max_resident", C.c_int), ("max_m", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("opts", DbOpts), ("gcv", DbGcvOpts)]


class DeblurError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

_VP = C.c_void_p
_SIGS = {
    "db_default_opts": (None, [C.POINTER(DbOpts), C.POINTER(DbGcvOpts)]),
    "db_context_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_size_t]),
    "db_context_destroy": (C.c_int, [_VP]),
    "db_last_error": (C.c_char_p, [_VP]),
    "db_footprint_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(DbGcvOpts)]),
    "deblur_solve": (C.c_int, [_VP, _VP, C.c_int, _VP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.POINTER(DbGcvOpts), C.POINTER(DbOpts), _VP, _VP, _VP, _VP, C.c_int, _VP]),
    "deblur_solve_batch": (C.c_int, [_VP, C.c_int, _VP, C.POINTER(DbGcvOpts), C.POINTER(DbOpts), C.c_int, _VP]),
    "db_server_create": (C.c_int, [_VP, C.POINTER(DbServerOpts), C.POINTER(_VP)]),
    "db_server_submit": (C.c_int, [_VP, C.POINTER(DbRequest), C.POINTER(C.c_uint64)]),
    "db_server_poll": (C.c_int, [_VP, C.c_uint64, C.c_int, C.POINTER(C.c_double)]),
    "db_server_cancel": (C.c_int, [_VP, C.c_uint64]),
    "db_server_destroy": (C.c_int, [_VP]),
    "db_set_profiling": (C.c_int, [_VP, C.c_int]),
    "db_set_autotune": (C.c_int, [_VP, C.c_int]),
    "db_get_stats": (C.c_int, [_VP, C.POINTER(DbStats)]),
    "db_reset_stats": (C.c_int, [_VP]),
    "db_apply_blur": (C.c_int, [_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_sumsq": (C.c_int, [_VP, C.c_size_t, C.c_int, C.POINTER(C.c_double), _VP]),
    "db_apply_L": (C.c_int, [C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_apply_Lt": (C.c_int, [C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_restrict": (C.c_int, [C.c_int, C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_prolong": (C.c_int, [C.c_int, C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_aux_prolong": (C.c_int, [C.c_int, C.c_int, _VP, _VP, C.c_int, _VP]),
    "db_lsqr_solve": (C.c_int, [_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_double, _VP, _VP, _VP, _VP, _VP,
                                C.POINTER(DbOpts), C.POINTER(C.c_int), C.c_int, _VP]),
    "db_lsqr_solve_static": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, C.c_double, _VP, _VP, _VP, _VP, _VP,
                                       C.POINTER(DbOpts), C.POINTER(C.c_int), C.c_int, _VP]),
    "db_gcv_select": (C.c_int, [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, C.POINTER(DbGcvOpts),
                                C.POINTER(C.c_double), C.c_int, _VP]),
}


def header_symbols():
    """Function names declared in include/deblur.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(db_\w+|deblur_\w+)\s*\(", txt)) - {"db_stream"})


def lib():
    """Load libdeblur.so once; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdeblur.so not built ({LIB_PATH}); run paper_2608_17123_b300/build.py")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_opts():
    o, g = DbOpts(), DbGcvOpts()
    lib().db_default_opts(C.byref(o), C.byref(g))
    return o, g


def check(status, ctx=None):
    if status != 0:
        msg = lib().db_last_error(ctx)
        raise DeblurError(status, msg.decode() if msg else "")
