"""Launch-shape autotuner for the solve kernels.

Times the self-scheduled (or level-scheduled) solve of a plan with CUDA
events on the current stream and keeps the fastest shape.  Two stages:
first the sub-warp width (lanes per row, hence rows per warp = 32 / lanes)
at the default block size, then, for that width, the block size and the cap
on the persistent grid (how many warps wait ahead of the dependency frontier:
more hides latency, fewer polls less L2 traffic).  Results are cached per
matrix signature for the process.
"""
from __future__ import annotations

import statistics

import torch

_CACHE: dict = {}

LANES = (1, 2, 4, 8, 16, 32)
BLOCKS = (128, 256, 512)
GRID_FRACTIONS = (0, 4, 2, 1)      # max_blocks = fraction * SMs (0: as many as fit)


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


def tune(plan, b, x=None, algo="self", lanes=LANES, blocks=BLOCKS, grids=GRID_FRACTIONS,
         reps=3, use_cache=True, transpose=False):
    """Pick lanes-per-row, block size and grid cap for `plan` on `b`.

    Sets the winner on the plan and returns ``{"best": (lanes, block,
    max_blocks, ms), "table": [(lanes, block, max_blocks, ms), ...]}``."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    key = signature(plan, nrhs, algo) + (transpose, tuple(lanes), tuple(blocks), tuple(grids))
    if use_cache and key in _CACHE:
        best = _CACHE[key]["best"]
        plan.set_tuning(best[0], best[1], best[2])
        return _CACHE[key]
    if x is None:
        x = torch.empty_like(b)
    sms = torch.cuda.get_device_properties(b.device).multi_processor_count
    table = []

    def run(w, blk, mb):
        plan.set_tuning(w, blk, mb)
        ms = time_solve(plan, b, x, algo, reps, transpose)
        table.append((w, blk, mb, ms))
        return ms

    default_block = 256 if 256 in blocks else blocks[0]
    for w in lanes:
        run(w, default_block, 0)
    w_best = min(table, key=lambda r: r[3])[0]
    if algo == "self":
        for blk in blocks:
            for frac in grids:
                if (blk, frac) != (default_block, 0):
                    run(w_best, blk, frac * sms)
    best = min(table, key=lambda r: r[3])
    plan.set_tuning(best[0], best[1], best[2])
    result = {"best": best, "table": table}
    _CACHE[key] = result
    return result
