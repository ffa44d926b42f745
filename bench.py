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


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("solve_self.cu", "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1710_04985_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(sha):
    """DRAM bytes per launch of the self-scheduled kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "self_solve_k1_ilu0_7pt_128.md")
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
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": pairs, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / pairs, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": L.n, "nnz_per_factor": L.nnz,
                       "step": "y = U^-1 (L^-1 b)", "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{pairs} L+U pairs of the full 128^3 factors, "
                                       "sequential FP64 oracle, one host thread"},
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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import synth
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
    b = torch.tensor(b_host, device=dev)
    y = torch.empty_like(b)
    x = torch.empty_like(b)
    tune_l = autotune.tune(pl, b, y)["best"]
    tune_u = autotune.tune(pu, y, x)["best"]

    def step(algo="self"):
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
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    kl_ms, kl_n = pl.profile_read()
    ku_ms, ku_n = pu.profile_read()
    pl.profile(False)
    pu.profile(False)
    launches = args.steps * 4
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    solves = 2 * args.steps * world
    value = solves / (ms / 1e3)
    bytes_solve = effective_bytes(n, nnz)
    kernel_avg_ms = (kl_ms + ku_ms) / max(1, kl_n + ku_n)
    peak, peak_kind = measured_peak_gbs()
    achieved = bytes_solve / (kernel_avg_ms / 1e3) / 1e9
    sha = kernel_source_sha()
    traffic = ncu_traffic(sha)

    # ---------------- end to end through the public API with host buffers
    hb = torch.tensor(b_host).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db, dy, dx = torch.empty_like(b), torch.empty_like(b), torch.empty_like(b)
    e2e_steps = max(3, min(args.steps, 100))

    def e2e_step():
        db.copy_(hb, non_blocking=True)
        pl.solve(db, out=dy)
        pu.solve(dy, out=dx)
        hx.copy_(dx, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = 2 * e2e_steps * world / e2e_s
    e2e_err = float(np.max(np.abs(hx.numpy() - xt)) / np.max(np.abs(xt)))

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
        extra["level_scheduled"] = {"solves_per_s": 2e3 / lv_ms, "ms_per_step": lv_ms,
                                    "effective_gbs": 2 * bytes_solve / (lv_ms / 1e3) / 1e9,
                                    "launches_per_step": 2 * 382}
        extra["cusparse_spsv"] = cusparse_pair(L, U, pl, pu, b, dev, lv_steps)
        self_ms = ms / args.steps
        extra["speedup_vs_level"] = lv_ms / self_ms
        if extra["cusparse_spsv"].get("ms_per_step"):
            extra["speedup_vs_cusparse"] = extra["cusparse_spsv"]["ms_per_step"] / self_ms

    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        pairs, el = time_oracle_pair(L, U, b_host, args.cpu_seconds)
        cpu = {"value": 2 * pairs / el, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"{pairs} L+U pairs of the full 128^3 factors "
                         f"({el:.1f} s, sequential FP64 oracle, one host thread)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "nnz_per_factor": nnz,
                       "nlev": [pl.levels()["nlev"], pu.levels()["nlev"]],
                       "step": "y = U^-1 (L^-1 b), eq. (3): 2 triangular solves",
                       "algo": "self-scheduled (Alg. 3)",
                       "tuning": {"L": list(tune_l[:3]), "U": list(tune_u[:3]),
                                  "fields": ["lanes_per_row", "block", "max_blocks"]},
                       "l2": "inputs larger than L2 (2 x 150 MB of matrix+vectors per step)",
                       "parallelism": f"replicas x{world}"},
            "effective_gbs": value / world * bytes_solve / 1e9 * world,
            "bytes_per_solve": bytes_solve,
            "roofline": {"bound": "hbm", "kernel": "self_solve_k1", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "traffic": traffic, "kernel_avg_ms": kernel_avg_ms,
                         "kernel_source_sha": sha},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": n * 8,
                    "d2h_bytes_per_step": n * 8, "steps": e2e_steps, "max_rel_err": e2e_err},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "analysis_ms": {"L": pl.analysis_ms, "U": pu.analysis_ms},
            "max_rel_err_vs_xtrue": err,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


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
    ref = pu.solve(pl.solve(b))
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
