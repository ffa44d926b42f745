"""Helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import torch

import oracle
import synth

# FP64 bar on max|x - x_ref| / max|x_ref|: the pull form reduces each row in a
# fixed order that differs from the sequential oracle's only in rounding, and the
# test matrices are well conditioned, so 1e-12 leaves several digits of margin.
TOL64 = 1e-12
# FP32 solves against the FP64 oracle: diagonally dominant / ILU factors keep
# the forward error within a small multiple of n_row * 2^-24.
TOL32 = 1e-4


def dev():
    return torch.device("cuda:0")


def tensors(A, dtype=torch.float64):
    d = dev()
    return (torch.tensor(A.rowptr, device=d), torch.tensor(A.colidx, device=d),
            torch.tensor(A.vals, device=d, dtype=dtype))


def plan_for(A, dtype=torch.float64, unit=None):
    from paper_1710_04985_gb300 import TriangularPlan
    rp, ci, va = tensors(A, dtype)
    return TriangularPlan(rp, ci, va, upper=A.upper, unit=A.unit if unit is None else unit)


def relerr(x, ref):
    x = x.detach().cpu().numpy() if isinstance(x, torch.Tensor) else x
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


def oracle_levels(A):
    lev, nlev = oracle.levels(A.rowptr, A.colidx, upper=A.upper)
    ilev, jlev = oracle.level_sets(lev, nlev)
    return lev, nlev, ilev, jlev


def assert_levels_equal(got, A, transpose=False):
    if transpose:
        lev, nlev = oracle.levels_transpose(A.rowptr, A.colidx, upper=A.upper)
        ilev, jlev = oracle.level_sets(lev, nlev)
    else:
        lev, nlev, ilev, jlev = oracle_levels(A)
    assert got["nlev"] == nlev
    assert np.array_equal(got["lev"].cpu().numpy(), lev)
    assert np.array_equal(got["ilev"].cpu().numpy(), ilev)
    assert np.array_equal(got["jlev"].cpu().numpy(), jlev)


def bidiagonal(n, upper=False):
    rows, cols = [], []
    for i in range(n):
        if upper:
            rows += [i] + ([i] if i + 1 < n else [])
            cols += [i] + ([i + 1] if i + 1 < n else [])
        else:
            rows += ([i] if i > 0 else []) + [i]
            cols += ([i - 1] if i > 0 else []) + [i]
    rows, cols = np.array(rows), np.array(cols)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    vals = np.where(rows == cols, 2.0, -0.5)
    return synth.CSR(n, rowptr, cols.astype(np.int32), vals, upper=upper, name=f"bidiag{n}")


def diagonal(n):
    rowptr = np.arange(n + 1, dtype=np.int32)
    colidx = np.arange(n, dtype=np.int32)
    return synth.CSR(n, rowptr, colidx, np.linspace(1.0, 3.0, n), name=f"diag{n}")


def long_rows(n=6000, seed=3):
    """Lower triangle whose rows include maximum-length (2000-entry) rows."""
    A = synth.general_lower(n, seed)
    rng = np.random.default_rng(seed)
    rows = A.row_of_entries().astype(np.int64)
    keys = rows * n + A.colidx
    extra = []
    for r in (2000, 2500, n - 1):
        cols = np.sort(rng.choice(r, 1999, replace=False))
        extra.append(r * n + cols)
    keys = np.unique(np.concatenate([keys] + extra))
    rr, cc = keys // n, keys % n
    # cap every row at 2000 entries keeping the diagonal
    keep = np.ones(keys.size, dtype=bool)
    starts = np.searchsorted(rr, np.arange(n))
    ends = np.searchsorted(rr, np.arange(n), side="right")
    for r in np.nonzero(ends - starts > 2000)[0]:
        keep[starts[r]:ends[r] - 2000] = False
    rr, cc = rr[keep], cc[keep]
    vals = np.where(rr == cc, 0.0, rng.uniform(-1, 1, rr.size))
    absum = np.bincount(rr[rr != cc], weights=np.abs(vals[rr != cc]), minlength=n)
    vals[rr == cc] = 1.0 + absum[rr[rr == cc]]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rr, minlength=n), out=rowptr[1:])
    return synth.CSR(n, rowptr, cc.astype(np.int32), vals, name="long_rows")


def unit_without_diagonal(n=3000, seed=4):
    """Unit-diagonal lower triangle whose diagonal is NOT stored (some rows
    are empty)."""
    A = synth.general_lower(n, seed)
    rows = A.row_of_entries()
    off = rows != A.colidx
    rr, cc = rows[off], A.colidx[off]
    vals = A.vals[off] / (1.0 + np.abs(A.vals[off]).sum())
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rr, minlength=n), out=rowptr[1:])
    return synth.CSR(n, rowptr, cc.astype(np.int32), vals, unit=True, name="unit_nodiag")
