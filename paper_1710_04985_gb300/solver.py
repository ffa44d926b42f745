"""Python face of the C ABI: a ``TriangularPlan`` holding one analysed sparse
triangular matrix (the setup phase of Sec. 4.4) and its solves.

PyTorch supplies device memory and streams only; every step runs in the CUDA
library through ``_lib``.  The plan borrows the CSR tensors given to it (it
keeps references so they stay alive).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import SptrsvError, check

ALGOS = {"level": _lib.ALGO_LEVEL, "self": _lib.ALGO_SELF, "tiled": _lib.ALGO_SELF_TILED,
         "chains": _lib.ALGO_SELF_CHAINS, "permuted": _lib.ALGO_SELF_PERMUTED,
         "column": _lib.ALGO_SELF_COLUMN, "blocked": _lib.ALGO_SELF_BLOCKED,
         "partitioned": _lib.ALGO_SELF_PARTITIONED}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class _DeviceArray:
    """Read-only view of plan-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _dev_int_array(ptr, n, device):
    if n == 0 or not ptr:
        return torch.zeros(0, dtype=torch.int32, device=device)
    return torch.as_tensor(_DeviceArray(ptr, n, "<i4"), device=device).clone()


def _need(t, name: str, dtype, device, fn: str):
    """A tensor the library reads or writes through a raw device pointer:
    its element type and device are those the call assumes (a host tensor
    or a narrower type would be read or written out of bounds on the GPU)."""
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or t.device != device:
        raise ValueError(f"{fn}: {name} must be a {dtype} tensor on {device}")


def _like(b: torch.Tensor):
    """An output with b's shape and strides (b already checked by
    _rhs_layout): residual and the refined solve take one leading dimension
    for their input and output arrays."""
    return torch.empty_strided(b.shape, b.stride(), dtype=b.dtype, device=b.device)


def _rhs_layout(t: torch.Tensor, n: int, name: str):
    """(nrhs, ld) of a row-major [n][ld] right-hand-side tensor."""
    if t.dim() == 1:
        if t.shape[0] != n or t.stride(0) != 1:
            raise ValueError(f"{name}: expected a contiguous vector of length {n}")
        return 1, 1
    if t.dim() != 2 or t.shape[0] != n or t.stride(1) != 1:
        raise ValueError(f"{name}: expected (n, k) with unit column stride, n = {n}")
    k = t.shape[1]
    ld = t.stride(0) if n > 1 else max(k, 1)
    if ld < k:
        raise ValueError(f"{name}: leading dimension {ld} < columns {k}")
    return k, ld


class TriangularPlan:
    """An analysed CSR triangular matrix, lower or upper, FP64 or FP32.

    ``rowptr``/``colidx`` are int32 CUDA tensors, ``vals`` float64 or
    float32, the diagonal stored in its row (ignored when ``unit``)."""

    def __init__(self, rowptr: torch.Tensor, colidx: torch.Tensor, vals: torch.Tensor,
                 upper: bool = False, unit: bool = False, stream=None):
        lib = _lib.load()
        for name, t, dt in (("rowptr", rowptr, torch.int32), ("colidx", colidx, torch.int32)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous int32 CUDA tensor")
        if vals.dtype not in (torch.float64, torch.float32) or not vals.is_cuda or \
                not vals.is_contiguous():
            raise ValueError("vals must be a contiguous float64/float32 CUDA tensor")
        if not rowptr.device == colidx.device == vals.device:
            raise ValueError("rowptr, colidx and vals must be on one device")
        self.n = rowptr.numel() - 1
        self.nnz = colidx.numel()
        if vals.numel() != self.nnz:
            raise ValueError("vals and colidx differ in length")
        self.dtype = vals.dtype
        self.upper = bool(upper)
        self.unit = bool(unit)
        self.device = vals.device
        self._keep = [rowptr, colidx, vals]
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = lib.sptrsv_analyze(
                self.n, self.nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                _lib.F64 if vals.dtype == torch.float64 else _lib.F32,
                _lib.UPPER if upper else _lib.LOWER, _lib.UNIT if unit else _lib.NON_UNIT,
                _stream_handle(stream), ctypes.byref(self._h))
        if st != _lib.OK:
            self._h = ctypes.c_void_p()
            check(st, "sptrsv_analyze", lib.sptrsv_last_error_row())

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().sptrsv_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def rowptr(self):
        return self._keep[0]

    @property
    def colidx(self):
        return self._keep[1]

    @property
    def vals(self):
        return self._keep[2]

    # ------------------------------------------------------------ solves
    @property
    def best_algo(self):
        """The form ``algo="auto"`` and the FP32 solves of ``solve_refined``
        run: the plan's default algorithm in the library (set by the
        autotuner; "self" until then)."""
        a = ctypes.c_int()
        check(_lib.load().sptrsv_get_default_algo(self._h, ctypes.byref(a)),
              "sptrsv_get_default_algo")
        return {v: k for k, v in ALGOS.items()}[a.value]

    @best_algo.setter
    def best_algo(self, name):
        check(_lib.load().sptrsv_set_default_algo(self._h, ALGOS[name]),
              "sptrsv_set_default_algo")

    best_algo_mrhs = "self"   # the multi-RHS form of algo="auto" (set by the autotuner)

    def _solve(self, fn, name, b, out, algo, stream):
        _need(b, "b", self.dtype, self.device, name)
        k, ld = _rhs_layout(b, self.n, "b")
        if algo == "auto":
            algo = self.best_algo if k == 1 else self.best_algo_mrhs
        if out is None:
            out = torch.empty_like(b, memory_format=torch.contiguous_format)
        _need(out, "out", self.dtype, self.device, name)
        k2, ld2 = _rhs_layout(out, self.n, "out")
        if k2 != k or ld2 != ld:
            raise ValueError(f"{name}: out must have the layout of b")
        check(fn(self._h, _ptr(b), _ptr(out), k, ld, ALGOS[algo], _stream_handle(stream)), name)
        return out

    def solve(self, b, out=None, algo="self", stream=None):
        """x = A^{-1} b (forward or backward substitution, Sec. 3.1).

        algo: "self" (Alg. 3, in place), "permuted" (on the level-ordered
        copy), "blocked" (tiles of that copy), "partitioned" (parts of
        consecutive rows, on the part-ordered copy), "tiled", "chains",
        "column" (Alg. 4), "level" (Alg. 1) or "auto" (the autotuner's
        choice, ``best_algo``)."""
        return self._solve(_lib.load().sptrsv_solve, "sptrsv_solve", b, out, algo, stream)

    def solve_transpose(self, b, out=None, algo="self", stream=None):
        """y = A^{-T} b (the CSC view of Sec. 3.2)."""
        return self._solve(_lib.load().sptrsv_solve_transpose, "sptrsv_solve_transpose", b,
                           out, algo, stream)

    def prepare_transpose(self, stream=None):
        check(_lib.load().sptrsv_prepare_transpose(self._h, _stream_handle(stream)),
              "sptrsv_prepare_transpose")

    def prepare(self, algo="auto", transpose=False, stream=None):
        """Build what the first solve of ``algo`` would build (copies,
        transposed pattern, segment order); synchronises.  Returns the host
        wall time in ms."""
        import time
        if algo == "auto":
            algo = self.best_algo
        t0 = time.perf_counter()
        check(_lib.load().sptrsv_prepare(self._h, int(bool(transpose)), ALGOS[algo],
                                         _stream_handle(stream)), "sptrsv_prepare")
        return 1e3 * (time.perf_counter() - t0)

    def grad_vals(self, y, x, out=None, stream=None):
        """-y_i . x_j on every stored (i, j): dloss/dA given y = A^{-T} dloss/dx."""
        _need(x, "x", self.dtype, self.device, "grad_vals")
        _need(y, "y", self.dtype, self.device, "grad_vals")
        k, ld = _rhs_layout(x, self.n, "x")
        ky, ldy = _rhs_layout(y, self.n, "y")
        if (k, ld) != (ky, ldy):
            raise ValueError("grad_vals: x and y must share their layout")
        if out is None:
            out = torch.empty(self.nnz, dtype=self.dtype, device=self.device)
        _need(out, "out", self.dtype, self.device, "grad_vals")
        if out.numel() != self.nnz or not out.is_contiguous():
            raise ValueError(f"grad_vals: out must be a contiguous vector of length {self.nnz}")
        check(_lib.load().sptrsv_grad_vals(self._h, _ptr(y), _ptr(x), k, ld, _ptr(out),
                                           _stream_handle(stream)), "sptrsv_grad_vals")
        return out

    def residual(self, b, x, out=None, stream=None):
        """r = b - A x in FP64."""
        for name, t in (("b", b), ("x", x)):
            _need(t, name, torch.float64, self.device, "residual")
        k, ld = _rhs_layout(b, self.n, "b")  # before _like(b): b's strides are valid
        if _rhs_layout(x, self.n, "x") != (k, ld):
            raise ValueError("residual: x must have the layout of b")
        if out is None:
            out = _like(b)
        _need(out, "out", torch.float64, self.device, "residual")
        if _rhs_layout(out, self.n, "out") != (k, ld):
            raise ValueError("residual: out must have the layout of b")
        check(_lib.load().sptrsv_residual(self._h, _ptr(b), _ptr(x), _ptr(out), k, ld,
                                          _stream_handle(stream)), "sptrsv_residual")
        return out

    def solve_refined(self, b, out=None, max_iter=10, tol=8 * 2.0 ** -52, stream=None):
        """FP32 bulk solves + FP64 residual/update iterative refinement.

        Returns ``(x, iterations, relative_residual)``."""
        _need(b, "b", torch.float64, self.device, "solve_refined")
        k, ld = _rhs_layout(b, self.n, "b")  # before _like(b): b's strides are valid
        if out is None:
            out = _like(b)
        _need(out, "out", torch.float64, self.device, "solve_refined")
        if _rhs_layout(out, self.n, "out") != (k, ld):
            raise ValueError("solve_refined: out must have the layout of b")
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        check(_lib.load().sptrsv_solve_refined(self._h, _ptr(b), _ptr(out), k, ld, max_iter,
                                               tol, ctypes.byref(it), ctypes.byref(rel),
                                               _stream_handle(stream)), "sptrsv_solve_refined")
        return out, it.value, rel.value

    REFINE_MODES = {"staged": _lib.REFINE_STAGED, "one_pass": _lib.REFINE_ONE_PASS}

    @property
    def refine_mode(self):
        """How ``solve_refined`` refines one right-hand side: "staged" (an
        FP32 solve pass and an FP64 residual pass per step) or "one_pass"
        (every step in one self-scheduled sweep)."""
        m = ctypes.c_int()
        check(_lib.load().sptrsv_get_refine_mode(self._h, ctypes.byref(m)),
              "sptrsv_get_refine_mode")
        return {v: k for k, v in self.REFINE_MODES.items()}[m.value]

    @refine_mode.setter
    def refine_mode(self, name):
        check(_lib.load().sptrsv_set_refine_mode(self._h, self.REFINE_MODES[name]),
              "sptrsv_set_refine_mode")

    def set_values(self, vals, stream=None):
        if vals.dtype != self.dtype or vals.device != self.device or \
                vals.numel() != self.nnz or not vals.is_contiguous():
            raise ValueError("set_values: same dtype, device and length, contiguous")
        check(_lib.load().sptrsv_set_values(self._h, _ptr(vals), _stream_handle(stream)),
              "sptrsv_set_values")
        self._keep[2] = vals

    def refresh_values(self, stream=None):
        check(_lib.load().sptrsv_refresh_values(self._h, _stream_handle(stream)),
              "sptrsv_refresh_values")

    ANALYSIS = {"sweep": _lib.ANALYSIS_SWEEP, "kahn_host_loop": _lib.ANALYSIS_KAHN_HOST_LOOP,
                "kahn_persistent": _lib.ANALYSIS_KAHN_PERSISTENT, "auto": _lib.ANALYSIS_AUTO}

    def reanalyze(self, method="auto", transpose=False, stream=None):
        """Recompute the levels of the forward (or transposed) system with
        ``method`` ("sweep", "kahn_host_loop" as in Sec. 4.4.1,
        "kahn_persistent", or "auto" as the plan's own setup); returns the
        analysis time in ms."""
        check(_lib.load().sptrsv_reanalyze(self._h, int(bool(transpose)), self.ANALYSIS[method],
                                           _stream_handle(stream)), "sptrsv_reanalyze")
        return self.analysis_ms

    def analysis_method(self, transpose=False):
        """Name of the analysis that produced the current levels."""
        m = ctypes.c_int()
        check(_lib.load().sptrsv_analysis_method(self._h, int(bool(transpose)),
                                                 ctypes.byref(m)), "sptrsv_analysis_method")
        return {v: k for k, v in self.ANALYSIS.items()}[m.value]

    # ------------------------------------------------------------ tuning
    def set_tuning(self, lanes_per_row, block_size=256, max_blocks=0):
        check(_lib.load().sptrsv_set_tuning(self._h, lanes_per_row, block_size, max_blocks),
              "sptrsv_set_tuning")

    def set_algo_tuning(self, algo, lanes_per_row=0, block_size=256, max_blocks=0):
        """Launch shape of one algorithm's single-RHS solves (lanes_per_row 0:
        use the plan's shape); ``set_tuning`` clears them all."""
        check(_lib.load().sptrsv_set_algo_tuning(self._h, ALGOS[algo], int(lanes_per_row),
                                                 int(block_size), int(max_blocks)),
              "sptrsv_set_algo_tuning")

    def set_mrhs_tuning(self, lanes_per_row=0, block_size=0, max_blocks=-1):
        """Launch shape of multi-RHS solves: width (0: one lane per column up
        to 16), block size (0) and grid cap (-1) default to the single-RHS
        ones."""
        check(_lib.load().sptrsv_set_mrhs_tuning(self._h, int(lanes_per_row), int(block_size),
                                                 int(max_blocks)), "sptrsv_set_mrhs_tuning")

    @property
    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(_lib.load().sptrsv_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)), "sptrsv_get_tuning")
        return {"lanes_per_row": a.value, "block_size": b.value, "max_blocks": c.value}

    def set_tiling(self, tile_rows, level_order=False):
        """Tiles of the tiled self-scheduled solve (algo="tiled"): runs of
        `tile_rows` consecutive positions of the substitution order, or of the
        level order when `level_order`."""
        check(_lib.load().sptrsv_set_tiling(self._h, int(tile_rows), int(bool(level_order))),
              "sptrsv_set_tiling")
        self._tiling = (int(tile_rows), bool(level_order))

    def set_tile_rows(self, tile_rows):
        self.set_tiling(tile_rows, self.tiling[1])

    @property
    def tiling(self):
        return getattr(self, "_tiling", (2048, False))

    def set_partition(self, part_rows=0, cluster_blocks=1):
        """Parts of the partitioned solve (algo="partitioned"): rows per part
        (0: the rows divided evenly over the SMs; reduced to what fits shared
        memory) and thread-block cluster size (1, 2, 4, 8: clusters read the
        values of their earlier parts in distributed shared memory)."""
        check(_lib.load().sptrsv_set_partition(self._h, int(part_rows), int(cluster_blocks)),
              "sptrsv_set_partition")

    @property
    def partition(self):
        """Rows per part the next partitioned solve uses."""
        return self.partition_shape[0]

    @property
    def partition_shape(self):
        """(rows per part, cluster blocks) of the next partitioned solve."""
        v, c = ctypes.c_int(), ctypes.c_int()
        check(_lib.load().sptrsv_get_partition(self._h, ctypes.byref(v), ctypes.byref(c)),
              "sptrsv_get_partition")
        return v.value, c.value

    def partition_info(self, transpose=False):
        """Layout of the partitioned solve's copy (after a partitioned solve in
        that direction): dict(nparts, nblocks, max_part_rows, part_ptr, order)
        with part_ptr[nparts + 1] the first position of every part in
        hand-out order and order[n] the row at every position."""
        np_, nb, mx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pp, od = ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.load().sptrsv_partition_info(self._h, int(bool(transpose)),
                                                ctypes.byref(np_), ctypes.byref(nb),
                                                ctypes.byref(mx), ctypes.byref(pp),
                                                ctypes.byref(od)), "sptrsv_partition_info")
        torch.cuda.synchronize(self.device)
        return {"nparts": np_.value, "nblocks": nb.value, "max_part_rows": mx.value,
                "part_ptr": _dev_int_array(pp.value, np_.value + 1 if self.n else 0, self.device),
                "order": _dev_int_array(od.value, self.n, self.device)}

    def set_spin_limit(self, polls):
        check(_lib.load().sptrsv_set_spin_limit(self._h, int(polls)), "sptrsv_set_spin_limit")

    def withhold_row(self, row):
        """Test hook: never publish ``row`` in self-scheduled solves (-1: off)."""
        check(_lib.load().sptrsv_debug_withhold_row(self._h, int(row)),
              "sptrsv_debug_withhold_row")

    # ------------------------------------------------------------ inspection
    def levels(self, transpose=False):
        """dict(nlev, lev, ilev, jlev) of the forward or transposed sweep."""
        nlev = ctypes.c_int()
        lev, ilev, jlev = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.load().sptrsv_levels(self._h, int(transpose), ctypes.byref(nlev),
                                        ctypes.byref(lev), ctypes.byref(ilev),
                                        ctypes.byref(jlev)), "sptrsv_levels")
        torch.cuda.synchronize(self.device)
        return {"nlev": nlev.value,
                "lev": _dev_int_array(lev.value, self.n, self.device),
                "ilev": _dev_int_array(ilev.value, nlev.value + 1 if self.n else 0, self.device),
                "jlev": _dev_int_array(jlev.value, self.n, self.device)}

    def transpose_pattern(self):
        a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.load().sptrsv_transpose_pattern(self._h, ctypes.byref(a), ctypes.byref(b),
                                                   ctypes.byref(c)), "sptrsv_transpose_pattern")
        torch.cuda.synchronize(self.device)
        return (_dev_int_array(a.value, self.n + 1, self.device),
                _dev_int_array(b.value, self.nnz, self.device),
                _dev_int_array(c.value, self.nnz, self.device))

    def status(self, stream=None):
        """(status code, row) of the first device-side failure since the last
        call; synchronises the stream and clears the record."""
        row = ctypes.c_int(-1)
        st = _lib.load().sptrsv_status(self._h, _stream_handle(stream), ctypes.byref(row))
        return st, row.value

    def check_status(self, stream=None):
        st, row = self.status(stream)
        check(st, "device status", row)

    @property
    def analysis_ms(self):
        v = ctypes.c_double()
        check(_lib.load().sptrsv_analysis_ms(self._h, ctypes.byref(v)), "sptrsv_analysis_ms")
        return v.value

    @property
    def last_launch_count(self):
        return _lib.load().sptrsv_last_launch_count(self._h)

    def profile(self, enable=True):
        check(_lib.load().sptrsv_profile_enable(self._h, int(bool(enable))),
              "sptrsv_profile_enable")

    def profile_read(self):
        """(total ms, solves timed) since the last read."""
        ms, cnt = ctypes.c_double(), ctypes.c_int()
        check(_lib.load().sptrsv_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt)),
              "sptrsv_profile_read")
        return ms.value, cnt.value


def plan_from_arrays(rowptr, colidx, vals, upper=False, unit=False, device="cuda",
                     dtype=torch.float64):
    """Copies host arrays (numpy or torch) to the device and analyses them."""
    rp = torch.as_tensor(rowptr, dtype=torch.int32).to(device).contiguous()
    ci = torch.as_tensor(colidx, dtype=torch.int32).to(device).contiguous()
    va = torch.as_tensor(vals).to(device=device, dtype=dtype).contiguous()
    return TriangularPlan(rp, ci, va, upper=upper, unit=unit)


__all__ = ["TriangularPlan", "plan_from_arrays", "SptrsvError"]
