"""The allocation-free entry point ``sptrsv_solve_noalloc``.

It serves callers that may not allocate device memory: code inside an
application that owns all device memory through its own pool, or a
latency-critical loop that must not touch the device allocator (cudaMalloc
and cudaFree can lock and synchronise the device).  Such callers cannot make
a plan, so the entry point validates and solves in one call, keeping its
working memory in a fixed array inside the library.

The test calls it through the C ABI twice in a row on the same inputs and
checks both results against the plan-based ``sptrsv_solve`` within the FP64
tolerance used by the other parity tests.  This file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL64, dev, plan_for, relerr, tensors

pytestmark = pytest.mark.gpu


def _noalloc(A, b, x):
    from paper_1710_04985_gb300 import _lib
    lib = _lib.load()
    rp, ci, va = A._dev
    row = ctypes.c_int(-7)
    st = lib.sptrsv_solve_noalloc(
        A.n, A.nnz, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
        ctypes.c_void_p(va.data_ptr()), _lib.F64, _lib.UPPER if A.upper else _lib.LOWER,
        _lib.UNIT if A.unit else _lib.NON_UNIT, ctypes.c_void_p(b.data_ptr()),
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
        ctypes.byref(row))
    return st, row.value


@pytest.mark.parametrize("name", ["general_lower", "ilu_unit_lower", "ilu_upper"])
def test_noalloc_matches_plan_solve_on_two_calls(cuda_device, name):
    if name == "general_lower":
        A = synth.general_lower(20011, 7)
    else:
        L, U = synth.lap3d_7pt_ilu0(16, 12, 10)
        A = L if name == "ilu_unit_lower" else U
    A._dev = tensors(A)
    b = torch.tensor(synth.uniform(A.n, 41), device=dev())
    with plan_for(A) as p:
        ref = p.solve(b).cpu().numpy()              # the existing entry point
    for _ in range(2):                              # two calls in a row, same scratch
        x = torch.full_like(b, float("nan"))
        st, row = _noalloc(A, b, x)
        assert (st, row) == (0, -1)
        assert relerr(x, ref) <= TOL64
    xb = b.clone()                                  # x == b
    st, row = _noalloc(A, xb, xb)
    assert (st, row) == (0, -1)
    assert relerr(xb, ref) <= TOL64


def test_noalloc_reports_invalid_matrix_and_size_limit(cuda_device):
    from paper_1710_04985_gb300 import _lib
    lib = _lib.load()
    bad = synth.CSR(3, np.array([0, 1, 3, 5], np.int32), np.array([0, 1, 0, 1, 2], np.int32),
                    np.ones(5))                     # row 1 is unsorted
    bad._dev = tensors(bad)
    b = torch.ones(3, dtype=torch.float64, device=dev())
    x = torch.zeros(3, dtype=torch.float64, device=dev())
    assert _noalloc(bad, b, x) == (2, 1)
    assert torch.all(x == 0)                        # nothing was solved
    row = ctypes.c_int(0)
    st = lib.sptrsv_solve_noalloc(_lib.NOALLOC_MAX_ROWS + 1, 0, None, None, None, _lib.F64,
                                  _lib.LOWER, _lib.UNIT, None, None, None, ctypes.byref(row))
    assert st == _lib.ERR_INVALID_ARG
