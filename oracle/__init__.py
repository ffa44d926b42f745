"""Sequential FP64 CPU oracle for sparse triangular solves.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
and its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``sptrsv_oracle.c`` (plain C, one loop per formula of
Li, arXiv:1710.04985, Secs. 3 and 4.1); this module only marshals numpy
arrays into it.  The shared library is compiled with gcc on first use (or by
``oracle.build.build()``).

Conventions: CSR with the diagonal stored in its row, 0-based int32 indices,
levels 0-based (the paper's level minus one), right-hand sides row-major
``(n, k)``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.library_path()
    if not os.path.exists(path) or _build.is_stale():
        _build.build()
    _lib = _bind(ctypes.CDLL(path))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded copy of the oracle library."""
    i, p_i, p_d = ctypes.c_int, _I32P, _F64P
    lib.oracle_levels_rowwise.argtypes = [i, p_i, p_i, i, p_i]
    lib.oracle_levels_rowwise.restype = i
    lib.oracle_levels_transpose.argtypes = [i, p_i, p_i, i, p_i]
    lib.oracle_levels_transpose.restype = i
    lib.oracle_level_sets.argtypes = [i, p_i, i, p_i, p_i]
    lib.oracle_level_sets.restype = None
    lib.oracle_solve.argtypes = [i, p_i, p_i, p_d, i, i, i, p_d, i, p_d, i]
    lib.oracle_solve.restype = None
    lib.oracle_solve_transpose.argtypes = [i, p_i, p_i, p_d, i, i, i, p_d, i, p_d, i]
    lib.oracle_solve_transpose.restype = None
    lib.oracle_grad_vals.argtypes = [i, p_i, p_i, i, i, p_d, i, p_d, i, p_d]
    lib.oracle_grad_vals.restype = None
    lib.oracle_residual.argtypes = [i, p_i, p_i, p_d, i, i, p_d, i, p_d, i, p_d, i]
    lib.oracle_residual.restype = None
    return lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _as2d(v):
    v = _f64(v)
    return (v.reshape(-1, 1), True) if v.ndim == 1 else (v, False)


def levels(rowptr, colidx, upper=False):
    """0-based level of every row by the row-wise loop of Sec. 4.1.

    Returns ``(lev, nlev)``."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    lev = np.zeros(n, dtype=np.int32)
    nlev = _load().oracle_levels_rowwise(n, rowptr, colidx, int(upper), lev)
    return lev, int(nlev)


def levels_transpose(rowptr, colidx, upper=False):
    """Levels of the transposed system A^T by the column-wise loop of Sec. 4.1
    (reading the CSR of A as the CSC of A^T).  Returns ``(lev, nlev)``."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    lev = np.zeros(n, dtype=np.int32)
    nlev = _load().oracle_levels_transpose(n, rowptr, colidx, int(upper), lev)
    return lev, int(nlev)


def level_sets(lev, nlev):
    """``(ilev, jlev)`` of Sec. 4.1: rows grouped by level, ascending row index
    within a level, ``ilev[m]`` the start of level m in ``jlev``."""
    lev = _i32(lev)
    n = len(lev)
    ilev = np.zeros(nlev + 1, dtype=np.int32)
    jlev = np.zeros(n, dtype=np.int32)
    _load().oracle_level_sets(n, lev, int(nlev), ilev, jlev)
    return ilev, jlev


def solve(rowptr, colidx, vals, b, upper=False, unit=False):
    """x = A^{-1} b by the row-wise substitution of Sec. 3.1 (reversed for
    upper triangles).  ``b`` is ``(n,)`` or ``(n, k)``."""
    rowptr, colidx, vals = _i32(rowptr), _i32(colidx), _f64(vals)
    b2, flat = _as2d(b)
    n, k = b2.shape
    x = np.zeros((n, k), dtype=np.float64)
    _load().oracle_solve(n, rowptr, colidx, vals, int(upper), int(unit), k,
                         b2, k, x, k)
    return x.reshape(-1) if flat else x


def solve_transpose(rowptr, colidx, vals, g, upper=False, unit=False):
    """y = A^{-T} g by the column-wise sweep of Sec. 3.2 on the CSR of A read
    as the CSC of A^T."""
    rowptr, colidx, vals = _i32(rowptr), _i32(colidx), _f64(vals)
    g2, flat = _as2d(g)
    n, k = g2.shape
    y = np.zeros((n, k), dtype=np.float64)
    _load().oracle_solve_transpose(n, rowptr, colidx, vals, int(upper),
                                   int(unit), k, g2, k, y, k)
    return y.reshape(-1) if flat else y


def grad_vals(rowptr, colidx, y, x, unit=False):
    """dloss/dA on the stored pattern: -y_i . x_j for every stored (i, j)
    (zero on the diagonal when ``unit``)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    y2, _ = _as2d(y)
    x2, _ = _as2d(x)
    n, k = x2.shape
    g = np.zeros(len(colidx), dtype=np.float64)
    _load().oracle_grad_vals(n, rowptr, colidx, int(unit), k, y2, k, x2, k, g)
    return g


def residual(rowptr, colidx, vals, b, x, unit=False):
    """r = b - A x (FP64)."""
    rowptr, colidx, vals = _i32(rowptr), _i32(colidx), _f64(vals)
    b2, flat = _as2d(b)
    x2, _ = _as2d(x)
    n, k = b2.shape
    r = np.zeros((n, k), dtype=np.float64)
    _load().oracle_residual(n, rowptr, colidx, vals, int(unit), k, b2, k,
                            x2, k, r, k)
    return r.reshape(-1) if flat else r
