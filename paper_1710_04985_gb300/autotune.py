"""Launch-shape autotuner for the solve kernels.

Times the solves of a plan with CUDA events on the current stream and keeps
the fastest shape.  ``tune`` searches one algorithm in two stages: first the
sub-warp width (lanes per row, hence rows per warp = 32 / lanes) at the
default block size, then, for that width, the block size and the cap on the
persistent grid (how many warps wait ahead of the dependency frontier: more
hides latency, fewer polls less L2 traffic), and for the tiled form the tile
size (for the partitioned form the part size).  ``tune_algos`` runs
``tune`` for the level-ordered (in place, on the level-ordered copy, and
blocked on that copy), partitioned, tiled and chained self-scheduled forms
and keeps the fastest, recording it on the plan.
Results are cached per matrix signature for the process.
"""
from __future__ import annotations

import statistics

import torch

_CACHE: dict = {}

LANES = (1, 2, 4, 8, 16, 32)
BLOCKS = (128, 256, 512)
GRID_FRACTIONS = (0, 4, 2, 1)      # max_blocks = fraction * SMs (0: as many as fit)
TILES = (1024, 2048, 4096)
PARTS = (0, 4096, 8192, 16384)     # rows per part of the partitioned form (0: automatic)
CLUSTERS = (2, 4)                  # thread-block cluster sizes tried for the partitioned form
TILED = ("tiled", "blocked", "partitioned")   # forms with a tile (or part) size
TILE_ORDERS = (False, True)      # substitution order, level order


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
         tiles=TILES, reps=3, use_cache=True, transpose=False, tile_orders=TILE_ORDERS,
         clusters=CLUSTERS):
    """Pick lanes-per-row, block size, grid cap (and tile size for "tiled")
    for `plan` on `b`.

    Sets the winner on the plan and returns ``{"best": (lanes, block,
    max_blocks, ms, tile_rows, level_order), "table": [...]}`` (for the
    partitioned form tile_rows is the part size and the last field the
    thread-block cluster size)."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    mrhs = nrhs > 1 and algo in ("self", "level", "permuted")
    if mrhs:
        # multi-RHS solves: the width is the multi-RHS one (4..32 lanes); one
        # lane per column at most
        cap = max(4, 1 << (nrhs - 1).bit_length())
        lanes = tuple(w for w in (4, 8, 16, 32) if w <= cap)
    key = signature(plan, nrhs, algo) + (transpose, tuple(lanes), tuple(blocks), tuple(grids),
                                         tuple(tiles), tuple(tile_orders))
    if use_cache and key in _CACHE:
        best = _CACHE[key]["best"]
        _apply(plan, best, algo, nrhs)
        return _CACHE[key]
    if x is None:
        x = torch.empty_like(b)
    sms = torch.cuda.get_device_properties(b.device).multi_processor_count
    esize = 8 if plan.dtype == torch.float64 else 4
    table = []

    tiles_used = algo in TILED

    def run(w, blk, mb, tile, order):
        if mrhs:
            plan.set_mrhs_tuning(w, blk, mb)
        else:
            plan.set_tuning(w, blk, mb)
        if algo == "partitioned":  # `order` holds the cluster size here
            plan.set_partition(tile, int(order) if order else 1)
        elif tiles_used:
            plan.set_tiling(tile, order)
        ms = time_solve(plan, b, x, algo, reps, transpose)
        table.append((w, blk, mb, ms, tile, order))
        return ms

    default_block = 256 if 256 in blocks else blocks[0]
    # the blocked form prefers small tiles (a tile should hold a few narrow levels)
    tile0 = min(tiles) if algo in ("blocked", "partitioned") else (2048 if 2048 in tiles
                                                                   else tiles[0])
    first_grid = 2 * sms if algo in ("tiled", "blocked") else 0
    orders = tile_orders if algo == "tiled" else (False,)
    # The blocked and partitioned forms hold a tile per block, so width and
    # block size interact (rows in flight per tile): with two block sizes or
    # fewer both are searched together in the first stage.
    joint = algo in ("blocked", "partitioned") and len(blocks) <= 2
    first_blocks = tuple(blocks) if joint else (default_block,)
    for order in orders:
        for w in lanes:
            for blk in first_blocks:
                run(w, blk, first_grid, tile0, order)
    w_best, order_best = min(table, key=lambda r: r[3])[0], min(table, key=lambda r: r[3])[5]
    if algo in ("self", "tiled", "chains", "permuted", "blocked", "partitioned"):
        for blk in blocks:
            for frac in grids:
                if (w_best, blk, frac * sms) not in {(r[0], r[1], r[2]) for r in table}:
                    run(w_best, blk, frac * sms, tile0, order_best)
    if tiles_used:
        bb = min(table, key=lambda r: r[3])
        for tile in tiles:
            # parts are reduced to what fits shared memory by the library
            if tile != tile0 and (algo == "partitioned" or tile * esize <= 48 * 1024 - 256):
                run(bb[0], bb[1], bb[2], tile, bb[5])
    if algo == "partitioned":
        bb = min(table, key=lambda r: r[3])
        for cl in clusters:
            run(bb[0], bb[1], bb[2], bb[4], cl)
    best = min(table, key=lambda r: r[3])
    _apply(plan, best, algo, nrhs)
    result = {"best": best, "table": table, "nrhs": nrhs}
    _CACHE[key] = result
    return result


def _apply(plan, best, algo, nrhs=1):
    """Set a tuning row on the plan: (lanes, block, max_blocks, ms, tile,
    level_order), lanes being the multi-RHS width when nrhs > 1."""
    if nrhs > 1 and algo in ("self", "level", "permuted"):
        plan.set_mrhs_tuning(best[0], best[1], best[2])
    else:
        plan.set_tuning(best[0], best[1], best[2])
    if algo == "partitioned":
        plan.set_partition(best[4], int(best[5]) if best[5] else 1)
    elif algo in ("tiled", "blocked"):
        plan.set_tiling(best[4], best[5])


# A small search per form (``tune_algos(..., quick=True)``): the shapes that
# won on the stencil factors, the general matrices and the batches measured
# so far, a few candidates each, for callers that tune several workloads in
# one short run.
QUICK = {
    # one or two blocks of 256 per SM: fewer polling warps win on deep, narrow
    # matrices (n = 10^6 general: 8 warps per SM 36.1 ms, 16: 39.1, all: 41.7)
    "self": dict(lanes=(1, 4, 8, 16, 32), blocks=(256,), grids=(0, 2, 1)),
    "permuted": dict(lanes=(1, 2, 4, 16), blocks=(256, 512), grids=(0, 1)),
    "blocked": dict(lanes=(1, 4), blocks=(512, 1024), grids=(0,), tiles=(256, 2048)),
    "partitioned": dict(lanes=(1, 2, 4, 8, 16), blocks=(512, 1024), grids=(0,),
                        tiles=(0, 8192, 16384), clusters=(4,)),
    "tiled": dict(lanes=(1, 4), blocks=(256,), grids=(0,), tiles=(2048,), tile_orders=(False,)),
    "chains": dict(lanes=(8, 16, 32), blocks=(256,), grids=(0, 2, 1)),
}


def tune_algos(plan, b, x=None, algos=("self", "permuted", "blocked", "partitioned", "tiled",
                                        "chains"), reps=3, use_cache=True, quick=False, **kw):
    """Tune each self-scheduled form and keep the faster one.

    Returns ``{"algo": name, "best": ..., "per_algo": {name: tune(...)}}`` and
    sets ``plan.best_algo`` (used by ``plan.solve(..., algo="auto")`` and by
    the FP32 solves of ``plan.solve_refined``).  ``quick``: the small
    per-form searches of ``QUICK``."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    if nrhs > 1:
        # multi-RHS solves run in place or on the level-ordered copy (the
        # blocked and partitioned forms use that copy too for nrhs > 1)
        algos = tuple(a for a in algos if a in ("self", "permuted")) or ("self",)
    per = {}
    for a in algos:
        if quick and not kw and nrhs == 1:
            per[a] = tune(plan, b, x, algo=a, reps=reps, use_cache=use_cache, **QUICK[a])
        elif a == "tiled" and not kw:
            # a lighter search: the tiled form wins only on chain-like matrices
            per[a] = tune(plan, b, x, algo=a, reps=reps, use_cache=use_cache, lanes=(1, 4, 16),
                          blocks=(256, 512), grids=(0, 2), tiles=(512, 2048))
        elif a == "blocked" and not kw:
            # narrow levels: large blocks cover a level or more
            per[a] = tune(plan, b, x, algo=a, reps=reps, use_cache=use_cache,
                          lanes=(1, 2, 4, 8), blocks=(512, 1024), grids=(0,),
                          tiles=(256, 512, 2048))
        elif a == "partitioned" and not kw:
            # parts of whole grid lines or planes; few lanes (short rows wait on
            # shared memory)
            per[a] = tune(plan, b, x, algo=a, reps=reps, use_cache=use_cache,
                          lanes=(1, 2, 4), blocks=(128, 256, 512), grids=(0,), tiles=PARTS)
        else:
            per[a] = tune(plan, b, x, algo=a, reps=reps, use_cache=use_cache, **kw)
    name = min(per, key=lambda a: per[a]["best"][3])
    _apply(plan, per[name]["best"], name, nrhs)
    if nrhs > 1:   # the multi-RHS form of algo="auto"
        plan.best_algo_mrhs = name
    else:
        plan.best_algo = name
        # every measured form keeps its own best shape (the FP32 solves of a
        # refined solve run the winning form, in its shape)
        for a, r in per.items():
            plan.set_algo_tuning(a, *r["best"][:3])
    return {"algo": name, "best": per[name]["best"], "per_algo": per}


def choice(result):
    """The winning (algo, lanes, block, max_blocks, tile_rows, level_order) of
    a ``tune_algos`` result, JSON-serialisable (for the partitioned form:
    part rows and cluster size in the last two)."""
    best = result["best"]
    last = int(best[5]) if result["algo"] == "partitioned" else bool(best[5])
    return [result["algo"], int(best[0]), int(best[1]), int(best[2]), int(best[4]), last]


def apply_choice(plan, ch):
    """Apply a ``choice`` to a plan without tuning; returns a result shaped
    like ``tune_algos``'s (no timing)."""
    algo, lanes, block, max_blocks, tile, order = ch
    best = (lanes, block, max_blocks, float("nan"), tile, order)
    _apply(plan, best, algo)
    plan.best_algo = algo
    return {"algo": algo, "best": best, "per_algo": {}}


def tune_refine(plan, b, reps=2):
    """Time ``plan.solve_refined(b)`` in both refinement forms (with the
    plan's current tuning), keep the faster one on the plan and return
    ``{"mode": name, "ms": {mode: ms}}``.  One right-hand side only (several
    always refine in the staged form)."""
    import time
    out = torch.empty_like(b)
    ms = {}
    for mode in ("staged", "one_pass"):
        plan.refine_mode = mode
        plan.solve_refined(b, out=out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            plan.solve_refined(b, out=out)
        torch.cuda.synchronize()
        ms[mode] = (time.perf_counter() - t0) / reps * 1e3
    best = min(ms, key=ms.get)
    plan.refine_mode = best
    return {"mode": best, "ms": ms}
