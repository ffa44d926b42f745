"""Benchmark: sparse triangular solves on one GB300 (or N replicas).

Workload (default): the ILU(0) factors L (unit lower) and U of the 3-D
7-point Laplacian on a 128^3 grid (n = 2,097,152, 8,339,456 stored entries
per factor, 382 levels each), FP64.  One step is the paper's solve pair
y = U^{-1} (L^{-1} b) (eq. (3)): a forward and a backward self-scheduled
solve.  ``value`` counts triangular solves per second over the whole job.

Beside it the same JSON line reports the level-scheduled solve (Alg. 1)
and cuSPARSE SpSV on the same data, the end-to-end rate through the public
API with host buffers, the roofline of the dominant kernel and the CPU
oracle timed on the host.

``--impl reference`` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import re
import statistics
import subprocess
import threading
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpTRSV solves/s & effective HBM GB/s vs plain level-set solve, same GB300"
WORKLOAD = "ilu0_7pt_128^3_LU_pair_fp64"
L2_BYTES = 129 * 2 ** 20


def effective_bytes(n, nnz, esize=8, nrhs=1):
    """Algorithmic HBM bytes of one triangular solve: value + column index per
    stored entry; row pointer + level-order index + b + x per row
    (nnz*12 + n*24 in FP64 for one right-hand side)."""
    return nnz * (esize + 4) + n * 8 + n * 2 * esize * nrhs


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Solve kernel of each self-scheduled form: (kernel name, source file, ncu
# summary of its launch on the 128^3 factor under profiles/, or None where no
# summary was taken: the roofline's traffic is then null)
KERNELS = {
    "self": ("self_solve_k1", "solve_self.cu", "self_solve_k1_ilu0_7pt_128.md"),
    "tiled": ("tiled_solve_k1", "solve_tiled.cu", None),
    "chains": ("chain_solve_k1", "solve_chain.cu", None),
    "permuted": ("self_solve_k1", "solve_self.cu", "self_solve_k1_permuted_ilu0_7pt_128.md"),
    "blocked": ("blocked_solve_k1", "solve_blocked.cu", None),
    "partitioned": ("blocked_solve_k1", "solve_blocked.cu",
                    "blocked_solve_k1_partitioned_ilu0_7pt_128.md"),
}


def _code_only(text):
    """Source text without comments and with whitespace collapsed, so that a
    comment edit does not count as a kernel change."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_sha(algo="self"):
    """Hash of the code (not the comments) of a solve kernel's source file and
    the shared headers: an ncu figure taken on other code is not reused."""
    h = hashlib.sha256()
    for f in (KERNELS[algo][1], "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1710_04985_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:12]


def ncu_traffic(sha, algo="self"):
    """DRAM bytes per launch of the solve kernel of `algo` from the committed
    ncu summary, if it was taken on the current kernel source."""
    if KERNELS[algo][2] is None:
        return None
    path = os.path.join(ROOT, "profiles", KERNELS[algo][2])
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*\(kernel source sha\s*([0-9a-f]+)\)",
                  text)
    if m and m.group(2) == sha:
        return float(m.group(1))
    return None


class ClockSampler:
    """nvidia-smi samples (every 100 ms) stamped on arrival with the host clock,
    so that a summary can be taken over any window: the timed region alone, or
    the whole measured phase (timed region, end-to-end and the other workloads).
    The sampler is live before the caller's first window opens."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.rows = []
        self.thread = None

    def _read(self):
        for line in self.proc.stdout:
            r = next(csv.reader([line]), [])
            if len(r) >= 9:
                self.rows.append((time.monotonic(), r))

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.monotonic() + 5.0
        while not self.rows and time.monotonic() < t_end and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0=None, t1=None, exclude=()):
        rows = [r for t, r in list(self.rows)
                if (t0 is None or t >= t0) and (t1 is None or t <= t1)
                and not any(a <= t <= b for a, b in exclude)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = sorted({self.NAMES[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, pg, device):
    """The slowest rank's elapsed milliseconds (every rank gets the result);
    with no process group, the local value."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processed `units_per_rank` units
    (weak scaling), in the slowest rank's `ms`."""
    return units_per_rank * world / (ms / 1e3)


def host_cpu():
    """Model name and logical core count of the host the CPU baseline ran on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(),
            "arch": platform.machine(), "nproc": os.cpu_count()}


def bench_config(n, nnz, nlev, world):
    """The workload description both arms print (the driver compares them)."""
    return {"workload": WORKLOAD, "n": n, "nnz_per_factor": nnz, "nlev": nlev,
            "step": "y = U^-1 (L^-1 b), eq. (3): 2 triangular solves",
            "l2": "inputs larger than L2 (2 x 150 MB of matrix+vectors per step)",
            "parallelism": f"replicas x{world}"}


def time_oracle_pair(L, U, b, budget_s, max_pairs=None):
    import oracle
    pairs, t0 = 0, time.perf_counter()
    while True:
        y = oracle.solve(L.rowptr, L.colidx, L.vals, b, unit=True)
        oracle.solve(U.rowptr, U.colidx, U.vals, y, upper=True)
        pairs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_pairs and pairs >= max_pairs):
            return pairs, el


def run_reference(args, world, rank):
    if rank != 0:
        return
    import synth
    L, U, xt, _, _ = synth.workload1()
    b = synth.times_vector(L, synth.times_vector(U, xt))
    time_oracle_pair(L, U, b, 0.0, max_pairs=args.warmup)
    pairs, el = time_oracle_pair(L, U, b, 1e9, max_pairs=args.steps)
    v = 2 * pairs / el
    import oracle
    nlev = [oracle.levels(A.rowptr, A.colidx, upper=A.upper)[1] for A in (L, U)]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": pairs, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / pairs, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(L.n, L.nnz, nlev, world),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{pairs} L+U pairs of the full 128^3 factors, "
                                       "sequential FP64 oracle, one host thread",
                             "host_cpu": host_cpu()},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--single-solve", choices=["L", "U", "G", "B"], default=None,
                    help="profiling target: build one plan (L or U factor of the 128^3 "
                         "ILU(0) workload, the n = 10^6 general matrix, or the 512-system "
                         "batch), apply --lanes/--max-blocks/--algo and run --repeat "
                         "solves (--refined: refined solves), nothing else")
    ap.add_argument("--refined", action="store_true",
                    help="--single-solve: FP32 + FP64 refined solves instead")
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--max-blocks", type=int, default=304)
    ap.add_argument("--algo", default="self",
                    choices=["self", "level", "tiled", "chains", "permuted", "column",
                             "blocked", "partitioned"])
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--part-rows", type=int, default=0,
                    help="--single-solve: rows per part of the partitioned form (0: automatic)")
    ap.add_argument("--cluster", type=int, default=1,
                    help="--single-solve: thread-block cluster size of the partitioned form")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other workload shapes (general matrix, multi-RHS, "
                         "refinement, autograd, 512-system batch)")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the headline line, print the Table 2 sweep: the solve "
                         "pair of eq. (3) on the 5/9-point 2-D and 7/27-point 3-D Laplacians "
                         "of every Table 2 grid, FP64 and FP32 (minutes)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuner choices: applied if it exists, written "
                         "after tuning otherwise (lets a profiler run reuse the plain run's "
                         "choices instead of re-tuning under the profiler)")
    ap.add_argument("--sweep-grids", type=int, default=5,
                    help="grids per stencil in --sweep (the first k of Table 2)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.single_solve:
        return single_solve(args)
    if args.sweep:
        return table2_sweep(args)

    import numpy as np

    import synth
    # host-side inputs first: the batch generator spawns worker processes
    W = None if args.headline_only else secondary_inputs()

    import torch

    from paper_1710_04985_gb300 import TriangularPlan, autotune

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    L, U, xt, _, _ = synth.workload1()
    b_host = synth.times_vector(L, synth.times_vector(U, xt))
    n, nnz = L.n, L.nnz

    def dplan(A):
        return TriangularPlan(torch.tensor(A.rowptr, device=dev), torch.tensor(A.colidx, device=dev),
                              torch.tensor(A.vals, device=dev), upper=A.upper, unit=A.unit)

    pl, pu = dplan(L), dplan(U)
    setup = {"L": pl.analysis_ms, "U": pu.analysis_ms,
             "method": [pl.analysis_method(), pu.analysis_method()],
             "note": "plan creation: validation, transposed pattern, levels "
                     "(SPTRSV_ANALYSIS_AUTO), level sets"}
    b = torch.tensor(b_host, device=dev)
    y = torch.empty_like(b)
    x = torch.empty_like(b)
    cached = None
    if args.tune_cache and os.path.exists(args.tune_cache):
        with open(args.tune_cache) as f:
            cached = json.load(f)
    if cached:
        tune_l = autotune.apply_choice(pl, cached["L"])
        tune_u = autotune.apply_choice(pu, cached["U"])
    else:
        tune_l = autotune.tune_algos(pl, b, y, reps=5)
        tune_u = autotune.tune_algos(pu, y, x, reps=5)
        if args.tune_cache:
            with open(args.tune_cache, "w") as f:
                json.dump({"L": autotune.choice(tune_l), "U": autotune.choice(tune_u)}, f)

    def step(algo="auto"):
        pl.solve(b, out=y, algo=algo)
        pu.solve(y, out=x, algo=algo)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    err = float(np.max(np.abs(x.cpu().numpy() - xt)) / np.max(np.abs(xt)))

    # ---------------- timed region: K steps, barrier + sync on both sides
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    pl.profile(True)
    pu.profile(True)
    pl.profile_read()
    pu.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local).__enter__()   # closed after the other workloads
    tt0 = time.monotonic()
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    tt1 = time.monotonic()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    kl_ms, kl_n = pl.profile_read()
    ku_ms, ku_n = pu.profile_read()
    pl.profile(False)
    pu.profile(False)
    launches = args.steps * (pl.last_launch_count + pu.last_launch_count)
    ms = max_over_ranks(ms, pg, dev)
    value = aggregate_rate(2 * args.steps, world, ms)
    bytes_solve = effective_bytes(n, nnz)
    kernel_avg_ms = (kl_ms + ku_ms) / max(1, kl_n + ku_n)
    peak, peak_kind = measured_peak_gbs()
    achieved = bytes_solve / (kernel_avg_ms / 1e3) / 1e9
    sha = kernel_source_sha(tune_l["algo"])
    traffic = ncu_traffic(sha, tune_l["algo"])

    # ---------------- end to end through the public API with host buffers
    hb = torch.tensor(b_host).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db, dy, dx = torch.empty_like(b), torch.empty_like(b), torch.empty_like(b)
    e2e_steps = max(3, min(args.steps, 100))

    def e2e_step():
        db.copy_(hb, non_blocking=True)
        pl.solve(db, out=dy, algo="auto")
        pu.solve(dy, out=dx, algo="auto")
        hx.copy_(dx, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_serial_s = time.perf_counter() - t0
    e2e_serial_err = float(np.max(np.abs(hx.numpy() - xt)) / np.max(np.abs(xt)))

    # The same steps pipelined the way a caller streaming right-hand sides
    # would run them: each step's H2D copy, its two solves and its D2H copy
    # are ordered by events on three streams (double-buffered device vectors),
    # so the copies of neighbouring steps overlap the latency-bound solves.
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    dbs = [torch.empty_like(b) for _ in range(2)]
    dxs = [torch.empty_like(b) for _ in range(2)]
    hxs = [torch.empty_like(hb).pin_memory() for _ in range(2)]
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "used", "out", "read")}

    def e2e_pipelined(steps):
        for k in range(steps):
            j = k % 2
            if k >= 2:
                s_in.wait_event(ev["used"][j])
            with torch.cuda.stream(s_in):
                dbs[j].copy_(hb, non_blocking=True)
            ev["in"][j].record(s_in)
            s_cmp.wait_event(ev["in"][j])
            if k >= 2:
                s_cmp.wait_event(ev["read"][j])
            pl.solve(dbs[j], out=dy, algo="auto", stream=s_cmp)
            ev["used"][j].record(s_cmp)
            pu.solve(dy, out=dxs[j], algo="auto", stream=s_cmp)
            ev["out"][j].record(s_cmp)
            s_out.wait_event(ev["out"][j])
            with torch.cuda.stream(s_out):
                hxs[j].copy_(dxs[j], non_blocking=True)
            ev["read"][j].record(s_out)

    torch.cuda.synchronize()
    e2e_pipelined(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_pipelined(e2e_steps)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = 2 * e2e_steps * world / e2e_s
    e2e_err = max(float(np.max(np.abs(h.numpy() - xt)) / np.max(np.abs(xt))) for h in hxs)

    extra = {}
    if not args.no_compare:
        # level-scheduled baseline (Alg. 1) on the same data, same tuning
        lv_steps = max(3, min(args.steps, 50))
        for _ in range(3):
            step("level")
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(lv_steps):
            step("level")
        a1.record()
        torch.cuda.synchronize()
        lv_ms = a0.elapsed_time(a1) / lv_steps
        # the same per-level launch sequence captured once in a CUDA graph
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step("level")
        lvg_ms = _events_ms(g.replay, lv_steps)
        extra["level_scheduled"] = {"solves_per_s": 2e3 / lv_ms, "ms_per_step": lv_ms,
                                    "effective_gbs": 2 * bytes_solve / (lv_ms / 1e3) / 1e9,
                                    "launches_per_step": 2 * 382,
                                    "graph_ms_per_step": lvg_ms,
                                    "graph_solves_per_s": 2e3 / lvg_ms}
        extra["cusparse_spsv"] = cusparse_pair(L, U, pl, pu, b, dev, lv_steps)
        self_ms = ms / args.steps
        # per-step distribution, back to back and with L2 flushed before every
        # step (a 2 x L2 memset outside the events)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
        dist_steps = {"back_to_back": [], "l2_flushed": []}
        for mode in dist_steps:
            for _ in range(50):
                if mode == "l2_flushed":
                    flush.zero_()
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                f0.record()
                step()
                f1.record()
                f1.synchronize()
                dist_steps[mode].append(f0.elapsed_time(f1))
        del flush
        extra["step_ms_distribution"] = {
            m: {"median": statistics.median(v), "mean": statistics.fmean(v), "min": min(v),
                "max": max(v), "steps": len(v)} for m, v in dist_steps.items()}
        # dependency-latency bound: a bidiagonal chain (n = 10^5, every row
        # waits on the previous one) gives the time of one dependency hop
        # t_hop; a solve of nlev levels cannot beat nlev * t_hop
        extra["latency_bound"] = chain_latency(dev, [pl.levels()["nlev"], pu.levels()["nlev"]],
                                               kernel_avg_ms)
        # setup phase (Sec. 4.4): the sync-free sweep against Kahn's algorithm
        # (Sec. 4.4.1), as the paper runs it (host loop) and in one persistent
        # launch; every method yields the same levels
        # the column-wise self-scheduled solve (Alg. 4, SLFC), the paper's
        # fastest on P100, tuned on its own and timed on the same pair
        kw = dict(lanes=(1, 2, 4, 8), blocks=(128, 256), grids=(0, 4, 2), reps=3)
        col_l = autotune.tune(pl, b, y, algo="column", **kw)
        col_u = autotune.tune(pu, y, x, algo="column", **kw)

        def col_step():
            pl.solve(b, out=y, algo="column")
            pu.solve(y, out=x, algo="column")

        col_ms = _events_ms(col_step, lv_steps)
        col_err = float(np.max(np.abs(x.cpu().numpy() - xt)) / np.max(np.abs(xt)))
        extra["column_wise_slfc"] = {"ms_per_step": col_ms, "solves_per_s": 2e3 / col_ms,
                                     "lanes": [col_l["best"][0], col_u["best"][0]],
                                     "row_wise_speedup": col_ms / self_ms,
                                     "max_rel_err_vs_xtrue": col_err}
        autotune.apply_choice(pl, autotune.choice(tune_l))
        autotune.apply_choice(pu, autotune.choice(tune_u))
        methods = {}
        for m in ("sweep", "kahn_host_loop", "kahn_persistent", "auto"):
            methods[m] = [pl.reanalyze(m), pu.reanalyze(m)]
        best_setup = sum(methods["auto"])
        extra["analysis_methods_ms"] = {"L_U": methods, "fields": "[L, U] wall ms, level "
                                        "analysis + level sets (+ transposed pattern for Kahn)"}
        cus = extra["cusparse_spsv"]
        if cus.get("ms_per_step"):
            # Sec. 5.2: smallest number of solve pairs n_s for which setup +
            # n_s solves beats cuSPARSE SpSV's setup + n_s solves
            extra["break_even_solves_vs_cusparse"] = _break_even(
                best_setup, self_ms, cus["analysis_ms_both"], cus["ms_per_step"])
        extra["speedup_vs_level"] = lv_ms / self_ms
        extra["speedup_vs_level_graph"] = lvg_ms / self_ms
        if extra["cusparse_spsv"].get("ms_per_step"):
            extra["speedup_vs_cusparse"] = extra["cusparse_spsv"]["ms_per_step"] / self_ms

    cpu, refs = None, None
    tc0 = tc1 = time.monotonic()
    if rank == 0 and args.cpu_seconds > 0:
        cpu, refs = cpu_leg(L, U, b_host, W, args.cpu_seconds)
        tc1 = time.monotonic()
    if W is not None:
        t_hop = (extra["latency_bound"]["t_hop_us"] if "latency_bound" in extra
                 else chain_latency(dev, [382], kernel_avg_ms)["t_hop_us"])
        extra.update(secondary(dev, W, refs, min(t_hop.values()), peak, pl, L))

    clk.__exit__(None, None, None)
    clocks = clk.summary(tt0 - 0.1, tt1 + 0.1)
    clocks["window"] = "timed region +- 100 ms (one sample period)"
    clocks["measured_phase"] = clk.summary(exclude=[(tc0, tc1)])
    clocks["measured_phase"]["window"] = ("timed region, end-to-end, comparisons and the "
                                          "other workloads (not the host-only oracle leg)")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(n, nnz, [pl.levels()["nlev"], pu.levels()["nlev"]], world),
            "tuning": {"algo": {"L": tune_l["algo"], "U": tune_u["algo"],
                                "self": "self-scheduled in level order (Alg. 3)",
                                "tiled": "self-scheduled over shared-memory tiles",
                                "chains": "self-scheduled over segments of consecutive "
                                          "rows, in-segment values passed by shuffle",
                                "permuted": "self-scheduled in level order on a level-ordered "
                                            "copy of the matrix (Sec. 4.3 remark 2)",
                                "blocked": "self-scheduled, a thread block per tile of the "
                                           "level-ordered copy, in-tile values in shared "
                                           "memory",
                                "partitioned": "self-scheduled, a thread block per part of "
                                               "consecutive rows (by level inside the part), "
                                               "in-part values in shared memory"},
                       "shape": {"L": _tuning_row(tune_l), "U": _tuning_row(tune_u),
                                 "fields": ["lanes_per_row", "block", "max_blocks",
                                            "tile_rows (part_rows when partitioned; 0: "
                                            "automatic)", "tile_level_order (cluster "
                                            "blocks when partitioned)"]}},
            "effective_gbs": value * bytes_solve / 1e9,
            # eq. (4): 2 nnz(A) / t for the pair, A = L + U - I (the 7-point operator)
            "gflops_eq4": 2 * (L.nnz + U.nnz - n) / (ms / args.steps / 1e3) / 1e9,
            "bytes_per_solve": bytes_solve,
            "roofline": {"bound": "hbm",
                         "kernel": KERNELS[tune_l["algo"]][0],
                         "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "traffic": traffic, "kernel_avg_ms": kernel_avg_ms,
                         "kernel_source_sha": sha},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": n * 8,
                    "d2h_bytes_per_step": n * 8, "steps": e2e_steps, "max_rel_err": e2e_err,
                    "how": "public API, pinned host b -> device -> L solve -> U solve -> host "
                           "x every step; copies and solves on three streams ordered by "
                           "events, double-buffered (host wall clock)",
                    "serial_value": 2 * e2e_steps * world / e2e_serial_s,
                    "serial_max_rel_err": e2e_serial_err},
            "gpu_launches": launches,
            "clocks": clocks,
            "analysis_ms": setup,
            "max_rel_err_vs_xtrue": err,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def single_solve(args):
    """A fixed plan and launch shape, `repeat` solves: the target of ncu
    captures (the capture selects one of the solve launches)."""
    import numpy as np
    import torch

    import synth
    from paper_1710_04985_gb300 import TriangularPlan
    dev = torch.device("cuda", 0)
    if args.single_solve == "G":
        A, xt, bh = synth.workload2()
    elif args.single_solve == "B":
        mats = synth.batch_general_parallel(512, synth.SEED_BASE + 3)
        A = synth.block_diagonal(mats)
        xt = np.concatenate([synth.uniform(m.n, 7000 + s) for s, m in enumerate(mats)])
        bh = synth.times_vector(A, xt)
    else:
        L, U, xt, bL, bU = synth.workload1()
        A, bh = (L, bL) if args.single_solve == "L" else (U, bU)
    p = TriangularPlan(torch.tensor(A.rowptr, device=dev), torch.tensor(A.colidx, device=dev),
                       torch.tensor(A.vals, device=dev), upper=A.upper, unit=A.unit)
    p.set_tuning(args.lanes, args.block, args.max_blocks)
    p.set_partition(args.part_rows, args.cluster)
    b = torch.tensor(bh, device=dev)
    x = torch.empty_like(b)
    if args.refined:
        p.set_algo_tuning("permuted", args.lanes, args.block, args.max_blocks)
        p.best_algo = args.algo
    for _ in range(args.repeat):
        if args.refined:
            p.solve_refined(b, out=x)
        else:
            p.solve(b, out=x, algo=args.algo)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(x.cpu().numpy() - xt)) / np.max(np.abs(xt)))
    print(json.dumps({"single_solve": args.single_solve, "algo": args.algo, "lanes": args.lanes,
                      "block": args.block, "max_blocks": args.max_blocks,
                      "part_rows": p.partition, "cluster": p.partition_shape[1],
                      "max_rel_err_vs_xtrue": err}))


def table2_sweep(args):
    """Sec. 5.1: the solve pair y = (U+D)^{-1} (L+D)^{-1} b of eq. (3) on the
    5/9-point 2-D and 7/27-point 3-D Laplacians of the Table 2 grids (aspect
    ratios of eq. (5)), in FP64 and FP32, for the self-scheduled solve (tuned),
    the level-scheduled solve and cuSPARSE SpSV on the same arrays.  GFLOPS
    follows eq. (4): 2 nnz(A) / t for the pair.  b is manufactured from a
    seeded x_true, and each row reports the error of the solution."""
    import numpy as np
    import torch

    import synth
    from paper_1710_04985_gb300 import TriangularPlan, autotune
    dev = torch.device("cuda", 0)
    rows = []
    cases = [(dims, pts) for pts in (5, 9) for dims in synth.TABLE2_GRIDS_2D[:args.sweep_grids]]
    cases += [(dims, pts) for pts in (7, 27) for dims in synth.TABLE2_GRIDS_3D[:args.sweep_grids]]
    for dims, pts in cases:
        L, U = synth.laplacian_triangles(dims, pts)
        xt = synth.uniform(L.n, synth.SEED_BASE + 10 + pts)
        bh = synth.times_vector(L, synth.times_vector(U, xt))
        nnz_a = L.nnz + U.nnz - L.n
        for dtype, dname in ((torch.float64, "f64"), (torch.float32, "f32")):
            def dplan(A):
                return TriangularPlan(torch.tensor(A.rowptr, device=dev),
                                      torch.tensor(A.colidx, device=dev),
                                      torch.tensor(A.vals, device=dev, dtype=dtype),
                                      upper=A.upper, unit=A.unit)
            pl, pu = dplan(L), dplan(U)
            b = torch.tensor(bh, device=dev, dtype=dtype)
            y, x = torch.empty_like(b), torch.empty_like(b)
            def tune_pair_member(p, rhs, out):
                # the level-ordered forms over all widths, the blocked form over
                # the narrow ones it can win with; the fastest is applied
                t = autotune.tune_algos(p, rhs, out, algos=("self", "permuted"),
                                        lanes=(1, 2, 4, 8, 16), blocks=(256, 512),
                                        grids=(0, 2), reps=3)
                tb = autotune.tune(p, rhs, out, algo="blocked", lanes=(1, 2, 4, 8),
                                   blocks=(512, 1024), grids=(0,), tiles=(256, 512, 2048),
                                   reps=3)
                if tb["best"][3] < t["best"][3]:
                    t = {"algo": "blocked", "best": tb["best"]}
                tp = autotune.tune(p, rhs, out, algo="partitioned", lanes=(1, 2, 4),
                                   blocks=(128, 256, 512), grids=(0,), tiles=autotune.PARTS,
                                   reps=3)
                if tp["best"][3] < t["best"][3]:
                    t = {"algo": "partitioned", "best": tp["best"]}
                autotune.apply_choice(p, autotune.choice(t))
                return t

            tl = tune_pair_member(pl, b, y)
            pl.solve(b, out=y, algo="auto")
            tu = tune_pair_member(pu, y, x)

            def pair(algo):
                pl.solve(b, out=y, algo=algo)
                pu.solve(y, out=x, algo=algo)

            ms = _events_ms(lambda: pair("auto"), 10)
            err = float(np.max(np.abs(x.double().cpu().numpy() - xt)) / np.max(np.abs(xt)))
            lv_ms = _events_ms(lambda: pair("level"), 2)
            esz = 8 if dtype == torch.float64 else 4
            byts = effective_bytes(L.n, L.nnz, esz) + effective_bytes(U.n, U.nnz, esz)
            cl = cusparse_single(L, pl, b, dev)
            cu = cusparse_single(U, pu, y, dev)
            cus = cl + cu if cl is not None and cu is not None else None
            analysis = None
            if dtype == torch.float64:
                analysis = {m: pl.reanalyze(m) for m in ("sweep", "kahn_persistent", "auto")}
                analysis["auto_picks"] = pl.analysis_method()
            row = {"grid": "x".join(map(str, dims)), "points": pts, "dtype": dname,
                   "n": L.n, "nnz_A": nnz_a,
                   "aspect": dims[1] // dims[0] if len(dims) == 2 else dims[2] // dims[0],
                   "nlev": [pl.levels()["nlev"], pu.levels()["nlev"]],
                   "self_ms": ms, "gflops": 2 * nnz_a / (ms / 1e3) / 1e9,
                   "effective_gbs": byts / (ms / 1e3) / 1e9,
                   "us_per_level": 1e3 * ms / (pl.levels()["nlev"] + pu.levels()["nlev"]),
                   "level_ms": lv_ms, "speedup_vs_level": lv_ms / ms,
                   "cusparse_ms": cus, "speedup_vs_cusparse": (cus / ms) if cus else None,
                   "lanes": [tl["best"][0], tu["best"][0]], "algo": [tl["algo"], tu["algo"]],
                   "analysis_ms_L": analysis,
                   "max_rel_err_vs_xtrue": err}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            pl.close()
            pu.close()
    print(json.dumps({"sweep": "table2", "unit_note": "ms per solve pair (L then U)",
                      "rows": rows}), flush=True)


def chain_latency(dev, nlevs, kernel_avg_ms, n=100_000):
    """Time of one dependency hop of the self-scheduled solve, from a lower
    bidiagonal chain of n rows (nlev = n): with one row per warp (32 lanes)
    every hop is a handshake between warps through L2; with 32 rows per warp
    (1 lane) consecutive rows share a warp.  Returns the hop times and the
    bound nlev * t_hop for the given level counts."""
    import numpy as np
    import torch

    import synth
    from paper_1710_04985_gb300 import TriangularPlan
    rows = np.repeat(np.arange(n), 2)[1:]
    cols = np.concatenate(([0], np.stack([np.arange(n - 1), np.arange(1, n)], 1).ravel()))
    vals = np.where(rows == cols, 2.0, -1.0)
    A = synth._from_sorted_coo(n, rows, cols, vals, upper=False)
    p = TriangularPlan(torch.tensor(A.rowptr, device=dev), torch.tensor(A.colidx, device=dev),
                       torch.tensor(A.vals, device=dev))
    b = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    hops = {}
    for lanes in (32, 1):
        p.set_tuning(lanes, 256, 0)
        hops[f"lanes{lanes}"] = _events_ms(lambda: p.solve(b, out=x, algo="self"), 3) * 1e3 / n
    p.close()
    t_hop = min(hops.values())  # the faster hop: a bound the solve cannot beat
    bound_ms = [nl * t_hop / 1e3 for nl in nlevs]
    return {"t_hop_us": hops, "nlev": nlevs, "bound_ms_per_solve": bound_ms,
            "kernel_avg_ms": kernel_avg_ms,
            "frac_of_bound": (sum(bound_ms) / len(bound_ms)) / kernel_avg_ms,
            "how": "lower bidiagonal chain n = 1e5, FP64, self-scheduled in place; "
                   "t_hop = the faster of one row per warp (a hop between warps) and "
                   "32 rows per warp; frac = nlev * t_hop / measured kernel time"}


def _break_even(setup_a, solve_a, setup_b, solve_b):
    """Smallest n >= 0 with setup_a + n solve_a < setup_b + n solve_b (None
    if never)."""
    if setup_a < setup_b:
        return 0
    if solve_a >= solve_b:
        return None
    return int((setup_a - setup_b) // (solve_b - solve_a)) + 1


def _tuning_row(t):
    """lanes, block, max_blocks, tile (or part) rows, tile level order (or,
    partitioned, the cluster size)."""
    best = t["best"]
    sized = t["algo"] in ("tiled", "blocked", "partitioned")
    last = (bool(best[5]) if t["algo"] == "tiled"
            else (int(best[5]) or 1) if t["algo"] == "partitioned" else None)
    return [best[0], best[1], best[2], best[4] if sized else None, last]


def _events_ms(fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def secondary_inputs():
    """Host-side inputs of the other workload shapes: the n = 10^6 general
    lower triangle with its manufactured right-hand side, the 512-system
    batch (b_s = A_s x_true,s), right-hand sides for the refinement and the
    autograd loss.  Generated before the first GPU call (the batch generator
    spawns worker processes)."""
    import numpy as np

    import synth
    A, xt, bh = synth.workload2()
    mats = synth.batch_general_parallel(512, synth.SEED_BASE + 3)
    bxt = [synth.uniform(m.n, 7000 + s) for s, m in enumerate(mats)]
    bb = [synth.times_vector(m, x) for m, x in zip(mats, bxt)]
    return {"general": (A, xt, bh),
            "batch": (mats, np.concatenate(bxt), np.concatenate(bb)),
            "refine_b": {"ilu_L": synth.uniform(2097152, 3100),
                         "general_1M": synth.uniform(A.n, 3100)},
            "loss": (synth.uniform(A.n, synth.SEED_BASE + 4),
                     synth.uniform(A.n, synth.SEED_BASE + 5))}


def cpu_leg(L, U, b_host, W, budget_s):
    """The CPU baseline: the sequential FP64 oracle on one host thread, timed
    on a bounded sample of the headline workload (L+U pairs for about
    `budget_s` seconds) and once on each other workload.  Its solutions are
    the references the GPU results of those workloads are compared with."""
    import numpy as np

    import oracle
    pairs, el = time_oracle_pair(L, U, b_host, budget_s)
    per, refs = {}, {}
    if W is not None:
        A, _, bh = W["general"]
        t0 = time.perf_counter()
        refs["general"] = oracle.solve(A.rowptr, A.colidx, A.vals, bh)
        per["general_1M_solve"] = 1e3 * (time.perf_counter() - t0)
        mats, _, bcat = W["batch"]
        off = np.concatenate(([0], np.cumsum([m.n for m in mats])))
        t0 = time.perf_counter()
        refs["batch"] = np.concatenate([
            oracle.solve(m.rowptr, m.colidx, m.vals, bcat[off[s]:off[s + 1]])
            for s, m in enumerate(mats)])
        per["batch_512_solves"] = 1e3 * (time.perf_counter() - t0)
        rb = W["refine_b"]
        refs["refine_ilu_L"] = oracle.solve(L.rowptr, L.colidx, L.vals, rb["ilu_L"], unit=True)
        refs["refine_general_1M"] = oracle.solve(A.rowptr, A.colidx, A.vals, rb["general_1M"])
        bl, tl = W["loss"]
        t0 = time.perf_counter()
        xr = oracle.solve(A.rowptr, A.colidx, A.vals, bl)
        yr = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, xr - tl)
        refs["grad_vals"] = oracle.grad_vals(A.rowptr, A.colidx, yr, xr)
        refs["grad_b"] = yr
        per["autograd_general_1M_gradient"] = 1e3 * (time.perf_counter() - t0)
    cpu = {"value": 2 * pairs / el, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"{pairs} L+U pairs of the full 128^3 factors ({el:.1f} s, sequential "
                     "FP64 oracle, one host thread)",
           "host_cpu": host_cpu(), "per_workload_ms": per}
    return cpu, refs


def _ms_stats(fn, reps):
    """Median and mean of `reps` CUDA-event timed calls (after one warm-up)."""
    import torch
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), statistics.fmean(times)


def _relerr(x, ref):
    import numpy as np
    x = x.detach().double().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def secondary(dev, W, refs, t_hop_us, peak, pl, L):
    """The other workload shapes, each timed with CUDA events after a short
    autotuner search: the n = 10^6 general matrix (FP64 and FP32, against the
    level-scheduled solve and cuSPARSE), multi-RHS on the 128^3 L factor,
    FP32 + FP64 refinement, the autograd gradient, and the 512-system batch.
    Every figure comes with its effective GB/s, its fraction of the measured
    HBM peak and of the dependency-latency bound nlev x t_hop."""
    import numpy as np
    import torch

    import synth
    from paper_1710_04985_gb300 import (BatchedTriangularSolve, TriangularPlan, autotune,
                                        sparse_triangular_solve)

    def dplan(A, dtype=torch.float64):
        return TriangularPlan(torch.tensor(A.rowptr, device=dev),
                              torch.tensor(A.colidx, device=dev),
                              torch.tensor(A.vals, device=dev, dtype=dtype),
                              upper=A.upper, unit=A.unit)

    def bounds(ms, byts, nlev):
        gbs = byts / ms / 1e6
        bound = nlev * t_hop_us / 1e3
        return {"effective_gbs": gbs, "frac_of_hbm_peak": gbs / peak,
                "latency_bound_ms": bound, "frac_of_latency_bound": bound / ms}

    res = {}
    ref = lambda k: refs.get(k) if refs else None  # noqa: E731

    # ---- general lower triangle, n = 10^6, FP64 and FP32
    A, xt, bh = W["general"]
    gen = {"n": A.n, "nnz": A.nnz}
    t_start = time.perf_counter()
    for dtype, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        p = dplan(A, dtype)
        b = torch.tensor(bh, device=dev, dtype=dtype)
        x = torch.empty_like(b)
        t = autotune.tune_algos(p, b, x, reps=2, quick=True)
        med, mean = _ms_stats(lambda: p.solve(b, out=x, algo="auto"), 10)
        esz = 8 if dtype == torch.float64 else 4
        nlev = p.levels()["nlev"]
        r = {"ms": med, "mean_ms": mean, "solves_per_s": 1e3 / med, "nlev": nlev,
             "algo": t["algo"], "tuning": _tuning_row(t),
             **bounds(med, effective_bytes(A.n, A.nnz, esz), nlev),
             "max_rel_err_vs_xtrue": _relerr(x, xt)}
        if ref("general") is not None:
            r["max_rel_err_vs_oracle"] = _relerr(x, ref("general"))
        r["level_scheduled_ms"] = _events_ms(lambda: p.solve(b, out=x, algo="level"), 2)
        r["speedup_vs_level"] = r["level_scheduled_ms"] / med
        cus = cusparse_single(A, p, b, dev)
        r["cusparse_ms"] = cus
        r["speedup_vs_cusparse"] = cus / med if cus else None
        r["analysis_ms"] = p.analysis_ms
        gen[name] = r
        if dtype == torch.float64:
            gen_plan = p
        else:
            p.close()
    gen["wall_s"] = time.perf_counter() - t_start
    res["general_1M"] = gen

    # ---- multi-RHS on the 128^3 ILU L factor: k = 1, 8, 32
    mr = {}
    for k in (1, 8, 32):
        bk = torch.tensor(synth.uniform((L.n, k) if k > 1 else L.n, 3000 + k), device=dev)
        xk = torch.empty_like(bk)
        if k > 1:
            t = autotune.tune_algos(pl, bk, xk, reps=2)
            form, lanes = t["algo"], t["best"][0]
        else:
            form, lanes = pl.best_algo, None
        med, mean = _ms_stats(lambda: pl.solve(bk, out=xk, algo="auto"), 10)
        byts = L.nnz * 12 + L.n * 8 + L.n * 16 * k
        mr[f"k{k}"] = {"ms": med, "mean_ms": mean, "rhs_solves_per_s": k * 1e3 / med,
                       "effective_gbs": byts / med / 1e6,
                       "frac_of_hbm_peak": byts / med / 1e6 / peak,
                       "algo": form, "lanes_per_row": lanes}
    res["multi_rhs_ilu_L"] = mr

    # ---- FP32 bulk solves + FP64 refinement (the faster of the two forms)
    ir = {}
    for name, p, A2 in (("ilu_L", pl, L), ("general_1M", gen_plan, A)):
        b2 = torch.tensor(W["refine_b"][name], device=dev)
        out = torch.empty_like(b2)
        forms = autotune.tune_refine(p, b2)
        p.solve_refined(b2, out=out)
        torch.cuda.synchronize()
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            _, iters, rel = p.solve_refined(b2, out=out)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        f64_ms = _events_ms(lambda: p.solve(b2, algo="auto"), 5)
        r = {"ms": ms, "corrections": iters, "final_rel_residual": rel,
             "form": forms["mode"], "ms_by_form": forms["ms"], "fp32_form": p.best_algo,
             "plain_fp64_solve_ms": f64_ms, "vs_plain_fp64": ms / f64_ms,
             "how": "host wall clock around the call; staged: an FP32 solve pass of the "
                    "tuned form (corrections added into x as published) and an FP64 "
                    "residual pass per step; one_pass: every step in one self-scheduled "
                    "sweep over the level-ordered copy"}
        if ref("refine_" + name) is not None:
            r["max_rel_err_vs_fp64_oracle"] = _relerr(out, ref("refine_" + name))
        ir[name] = r
    res["refinement"] = ir

    # ---- autograd: forward + backward of 0.5 ||A^{-1} b - t||^2 (general matrix)
    bl, tl = W["loss"]
    v = torch.tensor(A.vals, device=dev).requires_grad_(True)
    bb = torch.tensor(bl, device=dev).requires_grad_(True)
    tt = torch.tensor(tl, device=dev)

    def fwd_bwd():
        v.grad = None
        bb.grad = None
        xx = sparse_triangular_solve(gen_plan, v, bb, algo="auto")
        (0.5 * ((xx - tt) ** 2).sum()).backward()

    med, mean = _ms_stats(fwd_bwd, 5)
    ag = {"fwd_bwd_ms": med, "mean_ms": mean, "algo": gen_plan.best_algo,
          "forward_solve_ms": _events_ms(lambda: gen_plan.solve(bb.detach(), algo="auto"), 3)}
    if ref("grad_b") is not None:
        ag["max_rel_err_grad_b_vs_oracle"] = _relerr(bb.grad, ref("grad_b"))
        ag["max_rel_err_grad_vals_vs_oracle"] = _relerr(v.grad, ref("grad_vals"))
    res["autograd_general_1M"] = ag
    gen_plan.close()

    # ---- 512 independent systems, one graph-replayed launch
    mats, bxt, bcat = W["batch"]
    t_start = time.perf_counter()
    bs = BatchedTriangularSolve([(m.rowptr, m.colidx, m.vals) for m in mats], tune=False)
    bdev = torch.tensor(bcat, device=dev)
    bs.b.copy_(bdev)
    t = autotune.tune_algos(bs.plan, bs.b, bs.x, reps=2, quick=True)
    bs.capture()
    med, mean = _ms_stats(bs.graph.replay, 10)
    xb = bs.x.clone()
    off = np.asarray(bs.offsets)
    lev = bs.plan.levels()["lev"].cpu().numpy()
    sys_nlev = np.maximum.reduceat(lev, off[:-1]) + 1
    n_b, nnz_b = int(off[-1]), int(sum(m.nnz for m in mats))
    info = bs.plan.partition_info() if t["algo"] == "partitioned" else None
    plans = [dplan(m) for m in mats]
    bvs = [bdev[off[s]:off[s + 1]] for s in range(len(mats))]
    sep_ms = _events_ms(lambda: [pp.solve(bv) for pp, bv in zip(plans, bvs)], 2)
    for pp in plans:
        pp.close()
    r = {"systems": len(mats), "n_total": n_b, "nnz_total": nnz_b, "graph_ms": med,
         "mean_ms": mean, "separate_solves_ms": sep_ms, "speedup_vs_separate": sep_ms / med,
         "algo": t["algo"], "tuning": _tuning_row(t), "nlev_max_system": int(sys_nlev.max()),
         **bounds(med, effective_bytes(n_b, nnz_b), int(sys_nlev.max())),
         "max_rel_err_vs_xtrue": _relerr(xb, bxt)}
    if info:
        r["parts"] = {"nparts": info["nparts"], "independent_blocks": info["nblocks"],
                      "max_part_rows": info["max_part_rows"]}
    if ref("batch") is not None:
        r["max_rel_err_vs_oracle"] = _relerr(xb, ref("batch"))
    forms = autotune.tune_refine(bs.plan, bdev, reps=1)
    bs.solve_refined(bdev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xr, iters, rel = bs.solve_refined(bdev)
    torch.cuda.synchronize()
    r["refined"] = {"ms": 1e3 * (time.perf_counter() - t0), "corrections": iters,
                    "final_rel_residual": rel, "form": forms["mode"],
                    "ms_by_form": forms["ms"], "fp32_form": bs.plan.best_algo}
    if ref("batch") is not None:
        r["refined"]["max_rel_err_vs_fp64_oracle"] = _relerr(xr, ref("batch"))
    r["wall_s"] = time.perf_counter() - t_start
    res["batch_512"] = r
    return res


def cusparse_single(A, p, b, dev):
    """cuSPARSE SpSV solve time (ms) of one triangular system on the plan's
    device arrays, or None if the wrapper is unavailable."""
    import ctypes

    import torch

    from paper_1710_04985_gb300 import build
    path = build.cusparse_ref_path()
    if not os.path.exists(path):
        return None
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.cusref_create.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp)]
    lib.cusref_solve.argtypes = [vp, vp, vp, vp]
    lib.cusref_destroy.argtypes = [vp]
    y = torch.empty_like(b)
    s = vp(torch.cuda.current_stream().cuda_stream)
    h = vp()
    f64 = 1 if b.dtype == torch.float64 else 0
    if lib.cusref_create(A.n, A.nnz, vp(p.rowptr.data_ptr()), vp(p.colidx.data_ptr()),
                         vp(p.vals.data_ptr()), f64, int(A.upper), int(A.unit),
                         vp(b.data_ptr()), vp(y.data_ptr()), s, ctypes.byref(h)):
        return None
    ms = _events_ms(lambda: lib.cusref_solve(h, vp(b.data_ptr()), vp(y.data_ptr()), s), 3)
    lib.cusref_destroy(h)
    return ms


def cusparse_pair(L, U, pl, pu, b, dev, steps):
    """cuSPARSE SpSV (comparison only) on the same device arrays."""
    import ctypes

    import torch

    from paper_1710_04985_gb300 import build
    path = build.cusparse_ref_path()
    if not os.path.exists(path):
        return {"unavailable": "cuSPARSE wrapper not built"}
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.cusref_create.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp)]
    lib.cusref_solve.argtypes = [vp, vp, vp, vp]
    lib.cusref_destroy.argtypes = [vp]
    y = torch.empty_like(b)
    x = torch.empty_like(b)
    s = vp(torch.cuda.current_stream().cuda_stream)
    hl, hu = vp(), vp()
    t0 = time.perf_counter()
    rc = lib.cusref_create(L.n, L.nnz, vp(pl.rowptr.data_ptr()), vp(pl.colidx.data_ptr()),
                           vp(pl.vals.data_ptr()), 1, 0, 1, vp(b.data_ptr()), vp(y.data_ptr()),
                           s, ctypes.byref(hl))
    rc = rc or lib.cusref_create(U.n, U.nnz, vp(pu.rowptr.data_ptr()), vp(pu.colidx.data_ptr()),
                                 vp(pu.vals.data_ptr()), 1, 1, 0, vp(y.data_ptr()),
                                 vp(x.data_ptr()), s, ctypes.byref(hu))
    torch.cuda.synchronize()
    analysis_ms = 1e3 * (time.perf_counter() - t0)
    if rc:
        return {"unavailable": f"cuSPARSE status {rc}"}

    def pair():
        lib.cusref_solve(hl, vp(b.data_ptr()), vp(y.data_ptr()), s)
        lib.cusref_solve(hu, vp(y.data_ptr()), vp(x.data_ptr()), s)

    for _ in range(3):
        pair()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        pair()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ref = pu.solve(pl.solve(b, algo="auto"), algo="auto")
    agree = float((x - ref).abs().max() / ref.abs().max())
    lib.cusref_destroy(hl)
    lib.cusref_destroy(hu)
    bytes_pair = 2 * effective_bytes(L.n, L.nnz)
    return {"solves_per_s": 2e3 / ms, "ms_per_step": ms,
            "effective_gbs": bytes_pair / (ms / 1e3) / 1e9,
            "analysis_ms_both": analysis_ms, "max_rel_diff_vs_ours": agree,
            "api": "cusparseSpSV (CUSPARSE_SPSV_ALG_DEFAULT)"}


if __name__ == "__main__":
    main()
