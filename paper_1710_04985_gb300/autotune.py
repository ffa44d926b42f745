"""Launch-shape autotuner for the solve kernels.

Times the self-scheduled (or level-scheduled) solve of a plan for each
candidate sub-warp width (lanes per row, hence rows per warp = 32 / lanes)
and block size with CUDA events on the current stream, and keeps the
fastest.  Results are cached per matrix signature for the process.
"""
from __future__ import annotations

import statistics

import torch

_CACHE: dict = {}

LANES = (1, 2, 4, 8, 16, 32)
BLOCKS = (128, 256, 512)


def signature(plan, nrhs, algo):
    return (plan.n, plan.nnz, plan.upper, plan.unit, str(plan.dtype), nrhs, algo,
            int(plan.rowptr.data_ptr()), int(plan.colidx.data_ptr()))


def time_solve(plan, b, x, algo="self", reps=3, transpose=False):
    """Median milliseconds of `reps` solves (after one warm-up)."""
    fn = plan.solve_transpose if transpose else plan.solve
    fn(b, out=x, algo=algo)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(b, out=x, algo=algo)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune(plan, b, x=None, algo="self", lanes=LANES, blocks=BLOCKS, reps=3, use_cache=True,
         transpose=False):
    """Pick lanes-per-row and block size for `plan` on right-hand side `b`.

    Sets the winner on the plan and returns ``{"best": (lanes, block, ms),
    "table": [(lanes, block, ms), ...]}``."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    key = signature(plan, nrhs, algo) + (transpose,)
    if use_cache and key in _CACHE:
        best = _CACHE[key]["best"]
        plan.set_tuning(best[0], best[1], 0)
        return _CACHE[key]
    if x is None:
        x = torch.empty_like(b)
    table = []
    for w in lanes:
        for blk in blocks:
            plan.set_tuning(w, blk, 0)
            ms = time_solve(plan, b, x, algo, reps, transpose)
            table.append((w, blk, ms))
    best = min(table, key=lambda r: r[2])
    plan.set_tuning(best[0], best[1], 0)
    result = {"best": best, "table": table}
    _CACHE[key] = result
    return result
