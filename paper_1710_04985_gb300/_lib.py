"""ctypes binding of the C ABI in ``include/sptrsv.h``.

Argument marshalling only.  The shared library must have been built
(``__graft_entry__.build()`` or ``python -m paper_1710_04985_gb300.build``);
there is no fallback: a missing library is an error.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK = 0
ERR_INVALID_ARG = 1
ERR_STRUCTURE = 2
ERR_ZERO_PIVOT = 3
ERR_CUDA = 4
ERR_OOM = 5
ERR_TIMEOUT = 6
ERR_NOT_SUPPORTED = 7
ERR_INTERNAL = 8

ANALYSIS_SWEEP, ANALYSIS_KAHN_HOST_LOOP, ANALYSIS_KAHN_PERSISTENT, ANALYSIS_AUTO = 0, 1, 2, 3
F64, F32 = 0, 1
REFINE_STAGED, REFINE_ONE_PASS = 0, 1
LOWER, UPPER = 0, 1
NON_UNIT, UNIT = 0, 1
(ALGO_LEVEL, ALGO_SELF, ALGO_SELF_TILED, ALGO_SELF_CHAINS, ALGO_SELF_PERMUTED,
 ALGO_SELF_COLUMN, ALGO_SELF_BLOCKED, ALGO_SELF_PARTITIONED, ALGO_AUTO) = 0, 1, 2, 3, 4, 5, 6, 7, 8

# (name, restype, argtypes) for every entry point of include/sptrsv.h
_c_int, _c_ll, _c_dbl = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
_vp, _pp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)
_ip, _dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)

SIGNATURES = [
    ("sptrsv_analyze", _c_int, [_c_int, _c_int, _vp, _vp, _vp, _c_int, _c_int, _c_int, _vp, _pp]),
    ("sptrsv_free", _c_int, [_vp]),
    ("sptrsv_reanalyze", _c_int, [_vp, _c_int, _c_int, _vp]),
    ("sptrsv_analysis_method", _c_int, [_vp, _c_int, _ip]),
    ("sptrsv_solve", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("sptrsv_solve_transpose", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("sptrsv_prepare_transpose", _c_int, [_vp, _vp]),
    ("sptrsv_prepare", _c_int, [_vp, _c_int, _c_int, _vp]),
    ("sptrsv_grad_vals", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp, _vp]),
    ("sptrsv_residual", _c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("sptrsv_solve_refined", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_dbl, _ip, _dp, _vp]),
    ("sptrsv_set_default_algo", _c_int, [_vp, _c_int]),
    ("sptrsv_set_refine_mode", _c_int, [_vp, _c_int]),
    ("sptrsv_get_refine_mode", _c_int, [_vp, _ip]),
    ("sptrsv_get_default_algo", _c_int, [_vp, _ip]),
    ("sptrsv_set_values", _c_int, [_vp, _vp, _vp]),
    ("sptrsv_refresh_values", _c_int, [_vp, _vp]),
    ("sptrsv_set_tuning", _c_int, [_vp, _c_int, _c_int, _c_int]),
    ("sptrsv_get_tuning", _c_int, [_vp, _ip, _ip, _ip]),
    ("sptrsv_set_mrhs_tuning", _c_int, [_vp, _c_int, _c_int, _c_int]),
    ("sptrsv_set_algo_tuning", _c_int, [_vp, _c_int, _c_int, _c_int, _c_int]),
    ("sptrsv_set_spin_limit", _c_int, [_vp, _c_ll]),
    ("sptrsv_set_tiling", _c_int, [_vp, _c_int, _c_int]),
    ("sptrsv_set_partition", _c_int, [_vp, _c_int, _c_int]),
    ("sptrsv_get_partition", _c_int, [_vp, _ip, _ip]),
    ("sptrsv_partition_info", _c_int, [_vp, _c_int, _ip, _ip, _ip, _pp, _pp]),
    ("sptrsv_levels", _c_int, [_vp, _c_int, _ip, _pp, _pp, _pp]),
    ("sptrsv_transpose_pattern", _c_int, [_vp, _pp, _pp, _pp]),
    ("sptrsv_status", _c_int, [_vp, _vp, _ip]),
    ("sptrsv_last_error_row", _c_int, []),
    ("sptrsv_status_string", ctypes.c_char_p, [_c_int]),
    ("sptrsv_last_cuda_error", ctypes.c_char_p, []),
    ("sptrsv_analysis_ms", _c_int, [_vp, _dp]),
    ("sptrsv_profile_enable", _c_int, [_vp, _c_int]),
    ("sptrsv_profile_read", _c_int, [_vp, _dp, _ip]),
    ("sptrsv_last_launch_count", _c_int, [_vp]),
    ("sptrsv_debug_withhold_row", _c_int, [_vp, _c_int]),
    ("sptrsv_solve_noalloc", _c_int, [_c_int, _c_int, _vp, _vp, _vp, _c_int, _c_int, _c_int,
                                      _vp, _vp, _vp, _ip]),
]

NOALLOC_MAX_ROWS = 4194304
MAX_SIZE = 2147483392   # SPTRSV_MAX_SIZE: largest n and nnz a plan accepts (2^31 - 256)

_lib = None


class SptrsvError(RuntimeError):
    """A non-OK status from the C ABI."""

    def __init__(self, status: int, where: str, row: int = -1, detail: str = ""):
        self.status = status
        self.row = row
        name = status_string(status) if _lib is not None else str(status)
        msg = f"{where}: {name}"
        if row >= 0:
            msg += f" (row {row})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)


def library_path() -> str:
    return _build.library_path()


def load():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library {path} is missing: build it with __graft_entry__.build() "
            "(no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().sptrsv_status_string(int(status)).decode()


def check(status: int, where: str, row: int = -1):
    if status != OK:
        detail = ""
        if status == ERR_CUDA or status == ERR_OOM:
            detail = load().sptrsv_last_cuda_error().decode()
        raise SptrsvError(status, where, row, detail)
