"""The allocation-free entry point ``sptrsv_solve_noalloc``.

It serves callers that may not allocate device memory: code inside an
application that owns all device memory through its own pool, or a
latency-critical loop that must not touch the device allocator (cudaMalloc
and cudaFree can lock and synchronise the device).  Such callers cannot make
a plan, so the entry point validates and solves in one call, keeping its
working memory in a fixed array inside the library.

The tests call it through the C ABI twice in a row on the same inputs and
check both results against the oracle (FP64 within 1e-12, FP32 within the
FP32 bar of the other parity tests) and against the plan-based
``sptrsv_solve``; free device memory and the torch allocator's counters must
not move across a warmed-up call.  A wait that runs out (a row withheld by
the test hook) must come back as SPTRSV_ERR_TIMEOUT with the waiting row.
This file is named so that pytest collects it last.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL32, TOL64, bidiagonal, dev, plan_for, relerr, tensors

pytestmark = pytest.mark.gpu


def _noalloc(A, b, x, dtype=torch.float64):
    from paper_1710_04985_gb300 import _lib
    lib = _lib.load()
    rp, ci, va = A._dev
    row = ctypes.c_int(-7)
    st = lib.sptrsv_solve_noalloc(
        A.n, A.nnz, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
        ctypes.c_void_p(va.data_ptr()), _lib.F64 if dtype == torch.float64 else _lib.F32,
        _lib.UPPER if A.upper else _lib.LOWER, _lib.UNIT if A.unit else _lib.NON_UNIT,
        ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(row))
    return st, row.value


def _matrix(name):
    if name == "general_lower":
        return synth.general_lower(20011, 7)
    L, U = synth.lap3d_7pt_ilu0(16, 12, 10)
    return L if name == "ilu_unit_lower" else U


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["general_lower", "ilu_unit_lower", "ilu_upper"])
def test_noalloc_matches_oracle_on_two_calls(cuda_device, name, dtype):
    A = _matrix(name)
    A._dev = tensors(A, dtype)
    tol = TOL64 if dtype == torch.float64 else TOL32
    bh = synth.uniform(A.n, 41)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, bh, upper=A.upper, unit=A.unit)
    b = torch.tensor(bh, device=dev(), dtype=dtype)
    with plan_for(A, dtype) as p:
        plan_x = p.solve(b).double().cpu().numpy()    # the existing entry point
    assert relerr(plan_x, ref) <= tol
    x = torch.full_like(b, float("nan"))
    assert _noalloc(A, b, x, dtype) == (0, -1)         # warm-up: first use on the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    segs0 = torch.cuda.memory_stats().get("segment.all.allocated", 0)
    for _ in range(2):                                 # two calls in a row, same scratch
        x.fill_(float("nan"))
        st, row = _noalloc(A, b, x, dtype)
        assert (st, row) == (0, -1)
        xs = x.cpu().numpy().astype(np.float64)        # host copy: no device allocation
        assert relerr(xs, ref) <= tol
        assert relerr(xs, plan_x) <= tol
    torch.cuda.synchronize()
    # neither the library nor torch reserved device memory during the calls
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("segment.all.allocated", 0) == segs0
    xb = b.clone()                                     # x == b
    assert _noalloc(A, xb, xb, dtype) == (0, -1)
    assert relerr(xb.double(), ref) <= tol


def test_noalloc_reports_a_wait_that_runs_out(cuda_device, monkeypatch):
    """Row 319 of a bidiagonal chain is never published to other warps (test
    hook); row 320, first row of the next ticket, waits for it until the
    spin limit, reports SPTRSV_ERR_TIMEOUT and goes on with NaN.  The next
    call without the hook is exact again."""
    A = bidiagonal(2000)
    A._dev = tensors(A)
    bh = synth.uniform(A.n, 43)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, bh)
    b = torch.tensor(bh, device=dev())
    monkeypatch.setenv("SPTRSV_SPIN_LIMIT", str(1 << 12))
    monkeypatch.setenv("SPTRSV_DEBUG_NOALLOC_WITHHOLD", "319")
    x = torch.full_like(b, float("nan"))
    assert _noalloc(A, b, x) == (6, 320)
    xs = x.cpu().numpy()
    assert relerr(xs[:319], ref[:319]) <= TOL64
    assert np.all(np.isnan(xs[320:]))
    monkeypatch.delenv("SPTRSV_DEBUG_NOALLOC_WITHHOLD")
    assert _noalloc(A, b, x) == (0, -1)
    assert relerr(x, ref) <= TOL64
    assert "SPTRSV_DEBUG_NOALLOC_WITHHOLD" not in os.environ


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
