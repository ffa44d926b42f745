"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Levels and level sets must match bit for bit; FP64 solves within
max|x - x_ref| / max|x_ref| <= 1e-12; FP32 solves within 1e-4 of the FP64
oracle.  Sizes span many tiles and ragged tails; edge cases cover empty,
single-row, diagonal (nlev = 1), bidiagonal (nlev = n), maximum-length rows
and unit diagonals that are not stored.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import (TOL32, TOL64, assert_levels_equal, bidiagonal, dev, diagonal, long_rows,
                      plan_for, relerr, tensors, unit_without_diagonal)

pytestmark = pytest.mark.gpu


def _ilu_small():
    return synth.lap3d_7pt_ilu0(16, 12, 10)


MATRICES = {
    "workload0": lambda: synth.workload0()[0],
    "ilu_L": lambda: _ilu_small()[0],
    "ilu_U": lambda: _ilu_small()[1],
    "general": lambda: synth.general_lower(20011, 7),
    "general_upper": lambda: synth.to_upper_by_reversal(synth.general_lower(9001, 8)),
    "bidiag": lambda: bidiagonal(3001),
    "bidiag_upper": lambda: bidiagonal(1777, upper=True),
    "diag": lambda: diagonal(5000),
    "long_rows": long_rows,
    "unit_nodiag": unit_without_diagonal,
    "lap2d_upper": lambda: synth.lap2d_5pt_upper(37, 29),
    # the 9- and 27-point stencils of Sec. 5.1 (Table 2), both triangles
    "lap2d_9pt": lambda: synth.laplacian_triangles((37, 29), 9)[0],
    "lap2d_9pt_upper": lambda: synth.laplacian_triangles((37, 29), 9)[1],
    "lap3d_27pt": lambda: synth.laplacian_triangles((13, 11, 9), 27)[0],
    "lap3d_27pt_upper": lambda: synth.laplacian_triangles((13, 11, 9), 27)[1],
}

_cache = {}

ALL_ALGOS = ("self", "level", "permuted", "blocked", "column", "tiled", "chains",
             "partitioned")


def mat(name):
    if name not in _cache:
        _cache[name] = MATRICES[name]()
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_device):
    yield


# ---------------------------------------------------------------- levels

@pytest.mark.parametrize("name", list(MATRICES))
def test_levels_bit_exact(name):
    A = mat(name)
    with plan_for(A) as p:
        assert_levels_equal(p.levels(), A)


@pytest.mark.parametrize("name", ["workload0", "ilu_L", "ilu_U", "general", "general_upper",
                                  "bidiag", "long_rows", "unit_nodiag"])
def test_transpose_levels_and_pattern(name):
    A = mat(name)
    with plan_for(A) as p:
        p.prepare_transpose()
        assert_levels_equal(p.levels(transpose=True), A, transpose=True)
        tptr, tidx, tmap = (t.cpu().numpy() for t in p.transpose_pattern())
        T = A.scipy().T.tocsr()
        T.sort_indices()
        assert np.array_equal(tptr, T.indptr)
        assert np.array_equal(tidx, T.indices)
        assert np.array_equal(A.vals[tmap], T.data)


def test_automatic_analysis_choice():
    """The plan's own setup (SPTRSV_ANALYSIS_AUTO) levels wide graphs with
    Kahn's algorithm in one launch and gives up on deep, narrow ones after
    256 levels, falling back to the sweep; the levels are the same."""
    widening = synth.laplacian_triangles((300, 300), 9)[0]   # 898 levels, widening slowly
    narrow = synth.laplacian_triangles((40, 2000), 5)[0]     # 2039 levels of <= 40 rows
    cases = (("ilu_L", "kahn_persistent"), ("lap3d_27pt", "kahn_persistent"),
             ("bidiag", "sweep"), ("bidiag_upper", "sweep"),
             (widening, "kahn_persistent"), (narrow, "sweep"))
    for name, want in cases:
        A = mat(name) if isinstance(name, str) else name
        name = name if isinstance(name, str) else A.name
        with plan_for(A) as p:
            assert p.analysis_method() == want, name
            assert_levels_equal(p.levels(), A)
            p.prepare_transpose()
            assert p.analysis_method(transpose=True) == want, name
            assert_levels_equal(p.levels(transpose=True), A, transpose=True)


def test_automatic_analysis_many_plans():
    """Many plans in a row, as the benchmark's batch comparison makes them:
    every automatic analysis (Kahn's launch with its narrow runs, or the
    sweep after the probe) must finish and give the oracle's levels."""
    sizes = synth.batch_sizes(48, 77, nmin=300, nmax=9000)
    for s_, nk in enumerate(sizes):
        A = synth.general_lower(int(nk), 500 + s_)
        with plan_for(A) as p:
            assert_levels_equal(p.levels(), A)
            assert p.status() == (0, -1)
    for dims in ((40, 7), (3, 500), (9, 9, 9)):    # wide, narrow, and in between
        A = synth.laplacian_triangles(dims, 9 if len(dims) == 2 else 27)[0]
        for method in ("auto", "kahn_persistent"):
            with plan_for(A) as p:
                p.reanalyze(method)
                assert_levels_equal(p.levels(), A)


@pytest.mark.parametrize("method", ["kahn_host_loop", "kahn_persistent", "sweep", "auto"])
@pytest.mark.parametrize("name", ["workload0", "ilu_L", "ilu_U", "general", "general_upper",
                                  "bidiag", "diag", "long_rows", "unit_nodiag", "lap3d_27pt"])
def test_reanalyze_methods_give_the_same_levels(name, method):
    """Sec. 4.4.1: Kahn's algorithm (host loop as in the paper, or one
    persistent launch) and the sync-free sweep give the same (unique) levels
    and level sets, forward and transposed, and solves stay exact."""
    A = mat(name)
    b = synth.uniform(A.n, 25)
    with plan_for(A) as p:
        assert p.reanalyze(method) > 0
        assert_levels_equal(p.levels(), A)
        bt = torch.tensor(b, device=dev())
        ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
        for algo in ("self", "permuted", "level"):
            assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
        p.reanalyze(method, transpose=True)
        assert_levels_equal(p.levels(transpose=True), A, transpose=True)
        reft = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
        assert relerr(p.solve_transpose(bt), reft) <= TOL64
        assert p.status() == (0, -1)


# ---------------------------------------------------------------- solves

@pytest.mark.parametrize("algo", ["self", "level", "tiled", "tiled_levels", "chains", "permuted",
                                  "column", "blocked", "partitioned"])
@pytest.mark.parametrize("name", list(MATRICES))
def test_solve_fp64(name, algo):
    A = mat(name)
    b = synth.uniform(A.n, 11)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
    with plan_for(A) as p:
        if algo == "tiled_levels":
            p.set_tiling(512, True)
            algo = "tiled"
        x = p.solve(torch.tensor(b, device=dev()), algo=algo)
        assert relerr(x, ref) <= TOL64
        assert p.status() == (0, -1)


@pytest.mark.parametrize("algo", ["self", "level", "tiled", "chains", "permuted", "column",
                                  "blocked", "partitioned"])
@pytest.mark.parametrize("name", ["general", "ilu_L", "ilu_U", "long_rows"])
def test_solve_fp32(name, algo):
    A = mat(name)
    b = synth.uniform(A.n, 12)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
    with plan_for(A, torch.float32) as p:
        x = p.solve(torch.tensor(b, device=dev(), dtype=torch.float32), algo=algo)
        assert relerr(x.double(), ref) <= TOL32


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("block", [64, 256, 1024])
def test_every_launch_shape(lanes, block):
    A = mat("general")
    b = synth.uniform(A.n, 13)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with plan_for(A) as p:
        p.set_tuning(lanes, block, 0)
        bt = torch.tensor(b, device=dev())
        for algo in ("self", "level", "chains", "permuted", "column", "partitioned"):
            assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
        p.set_tuning(lanes, block, 3)          # a tiny persistent grid still finishes
        assert relerr(p.solve(bt, algo="partitioned"), ref) <= TOL64
        assert relerr(p.solve(bt), ref) <= TOL64
        assert relerr(p.solve(bt, algo="chains"), ref) <= TOL64
        assert relerr(p.solve(bt, algo="permuted"), ref) <= TOL64
        assert relerr(p.solve(bt, algo="column"), ref) <= TOL64
        for order in (False, True):            # tiled form: ragged and largest tiles
            for tile in (32, 100, 2048, 6112):
                p.set_tiling(tile, order)
                assert relerr(p.solve(bt, algo="tiled"), ref) <= TOL64
                assert relerr(p.solve(bt, algo="blocked"), ref) <= TOL64


def test_per_algorithm_launch_shape():
    """sptrsv_set_algo_tuning gives one algorithm its own launch shape over the
    plan's; sptrsv_set_tuning clears every such override.  Widths 1 and 32
    fold a row in different trees, so the results show which shape ran."""
    from paper_1710_04985_gb300 import SptrsvError
    A = mat("general")
    b = synth.uniform(A.n, 28)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with plan_for(A) as p:
        bt = torch.tensor(b, device=dev())
        p.set_tuning(32, 1024, 3)
        w32 = p.solve(bt).clone()
        p.set_tuning(1, 128, 0)
        w1 = p.solve(bt).clone()
        assert relerr(w32, ref) <= TOL64 and relerr(w1, ref) <= TOL64
        assert not torch.equal(w1, w32)
        p.set_algo_tuning("self", 32, 1024, 3)
        assert torch.equal(p.solve(bt), w32)                   # its own shape
        assert torch.equal(p.solve(bt, algo="permuted"), w1)   # the plan's shape
        p.set_algo_tuning("permuted", 32, 256, 0)
        assert torch.equal(p.solve(bt, algo="permuted"), w32)
        p.set_algo_tuning("self", 0)                           # cleared: the plan's shape
        assert torch.equal(p.solve(bt), w1)
        p.set_tuning(1, 128, 0)                                # clears every override
        assert torch.equal(p.solve(bt, algo="permuted"), w1)
        for bad in ((3, 256, 0), (4, 48, 0), (4, 256, -1)):
            with pytest.raises(SptrsvError):
                p.set_algo_tuning("self", *bad)


@pytest.mark.parametrize("k", [2, 3, 8, 32, 33])
@pytest.mark.parametrize("algo", ["self", "level", "tiled", "chains", "permuted", "blocked",
                                  "partitioned"])
def test_multi_rhs(k, algo):
    """Every form takes several right-hand sides: the copying forms run the
    multi-RHS kernel on the level-ordered copy (bitwise equal to the
    in-place multi-RHS kernel: same width, same fold order per column), the
    others the in-place or level-scheduled multi-RHS kernel."""
    for name in ("general", "ilu_U", "ilu_L"):
        A = mat(name)
        b = synth.uniform((A.n, k), 14 + k)
        ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
        with plan_for(A) as p:
            bt = torch.tensor(b, device=dev())
            x = p.solve(bt, algo=algo)
            assert relerr(x, ref) <= TOL64
            if algo in ("permuted", "blocked", "partitioned"):
                assert torch.equal(x, p.solve(bt, algo="self"))
                reft = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, b, upper=A.upper,
                                              unit=A.unit)
                assert relerr(p.solve_transpose(bt, algo=algo), reft) <= TOL64
            assert p.status() == (0, -1)


def test_multi_rhs_width_does_not_change_results():
    """Every column is folded in entry order by one lane, so the multi-RHS
    width (lanes per row, several columns per lane when narrower than k)
    changes the schedule only: results are bitwise equal and exact."""
    from paper_1710_04985_gb300 import autotune
    A = mat("general")
    for k in (5, 33):
        b = synth.uniform((A.n, k), 40 + k)
        ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
        with plan_for(A) as p:
            bt = torch.tensor(b, device=dev())
            first = p.solve(bt).clone()
            assert relerr(first, ref) <= TOL64
            for w in (4, 8, 16, 32, 0):
                p.set_mrhs_tuning(w, 128 if w == 8 else 0, 76 if w == 16 else -1)
                assert torch.equal(p.solve(bt), first), (k, w)
                # the level-scheduled form uses the same width (and divides by
                # d(i) where the self-scheduled one multiplies by 1/d(i))
                assert relerr(p.solve(bt, algo="level"), ref) <= TOL64
            res = autotune.tune_algos(p, bt, use_cache=False, blocks=(256,), grids=(0, 2))
            assert res["best"][0] in (4, 8, 16, 32)
            assert torch.equal(p.solve(bt, algo="auto"), first)
    with plan_for(A) as p:
        from paper_1710_04985_gb300 import SptrsvError
        before = p.tuning
        for bad in ((3, 0, -1), (8, 48, -1), (8, 0, -2)):
            with pytest.raises(SptrsvError):
                p.set_mrhs_tuning(*bad)
        p.set_mrhs_tuning(16, 512, 4)
        assert p.tuning == before          # the single-RHS shape is left alone


@pytest.mark.parametrize("algo", ["self", "level", "tiled", "chains", "permuted", "column",
                                  "blocked", "partitioned"])
def test_leading_dimension_and_in_place(algo):
    A = mat("general")
    k, ld = 3, 5
    b = synth.uniform((A.n, k), 15)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with plan_for(A) as p:
        big = torch.zeros((A.n, ld), dtype=torch.float64, device=dev())
        big[:, :k] = torch.tensor(b, device=dev())
        out = torch.full((A.n, ld), 7.0, dtype=torch.float64, device=dev())
        p.solve(big[:, :k], out=out[:, :k], algo=algo)
        assert relerr(out[:, :k], ref) <= TOL64
        assert torch.all(out[:, k:] == 7.0)          # untouched padding columns
        inplace = big[:, :k]
        p.solve(inplace, out=inplace, algo=algo)      # x == b
        assert relerr(inplace, ref) <= TOL64
        v = torch.tensor(b[:, 0].copy(), device=dev())
        p.solve(v, out=v, algo=algo)
        assert relerr(v, ref[:, 0]) <= TOL64


@pytest.mark.parametrize("algo", ["self", "level", "tiled", "tiled_levels", "chains", "permuted",
                                  "column", "blocked", "partitioned"])
@pytest.mark.parametrize("name", ["workload0", "ilu_L", "ilu_U", "general", "general_upper",
                                  "long_rows", "unit_nodiag", "bidiag"])
def test_solve_transpose(name, algo):
    A = mat(name)
    level_tiles = algo == "tiled_levels"
    algo = "tiled" if level_tiles else algo
    for k in (1, 4):
        g = synth.uniform((A.n, k) if k > 1 else A.n, 16)
        ref = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, g, upper=A.upper, unit=A.unit)
        with plan_for(A) as p:
            if level_tiles:
                p.set_tiling(1000, True)
            y = p.solve_transpose(torch.tensor(g, device=dev()), algo=algo)
            assert relerr(y, ref) <= TOL64


@pytest.mark.parametrize("name", ["general", "general_upper", "ilu_U"])
def test_bitwise_determinism_and_algo_agreement(name):
    """The pull form fixes each row's reduction order (farthest dependency
    first: an upper row from its last entry back, in place and in every
    copy), so repeated solves agree bit for bit and so do the forms.  The
    level-scheduled form divides by d(i) (Alg. 1) and the self-scheduled one
    multiplies by 1/d(i) (as the paper's SLFR kernel does), so the two agree
    to rounding."""
    A = mat(name)
    with plan_for(A) as p:
        bt = torch.tensor(synth.uniform(A.n, 17), device=dev())
        first = p.solve(bt).clone()
        for _ in range(20):
            assert torch.equal(p.solve(bt), first)
        lv = p.solve(bt, algo="level")
        for _ in range(5):
            assert torch.equal(p.solve(bt, algo="level"), lv)
        assert relerr(lv, first.cpu().numpy()) <= 1e-14
        # the tiled and chained forms reduce each row in the same order as the
        # level-ordered one
        for order in (False, True):
            p.set_tiling(1024, order)
            for _ in range(3):
                assert torch.equal(p.solve(bt, algo="tiled"), first)
        for _ in range(3):
            assert torch.equal(p.solve(bt, algo="chains"), first)
        # so do the level-ordered copy, whose rows are stored in fold order,
        # and the blocked solve on it (any tile size)
        for _ in range(3):
            assert torch.equal(p.solve(bt, algo="permuted"), first)
        for tile in (64, 1000, 4096):
            p.set_tiling(tile, False)
            assert torch.equal(p.solve(bt, algo="blocked"), first)
        # and the partitioned solve, whatever the part size
        for rows in (0, 1, 77, 1000, A.n, 1 << 20):
            p.set_partition(rows)
            assert torch.equal(p.solve(bt, algo="partitioned"), first), rows
        tg = torch.tensor(synth.uniform(A.n, 23), device=dev())
        assert torch.equal(p.solve_transpose(tg, algo="permuted"), p.solve_transpose(tg))
        assert torch.equal(p.solve_transpose(tg, algo="partitioned"), p.solve_transpose(tg))
        # the column-wise form (Alg. 4) adds contributions atomically in
        # arrival order: equal to rounding only
        for _ in range(3):
            assert relerr(p.solve(bt, algo="column"), first.cpu().numpy()) <= 1e-13


# ---------------------------------------------------------------- edge cases

def test_empty_matrix():
    from paper_1710_04985_gb300 import TriangularPlan
    d = dev()
    p = TriangularPlan(torch.zeros(1, dtype=torch.int32, device=d),
                       torch.zeros(0, dtype=torch.int32, device=d),
                       torch.zeros(0, dtype=torch.float64, device=d))
    assert p.levels()["nlev"] == 0
    for algo in ALL_ALGOS:
        out = p.solve(torch.zeros(0, dtype=torch.float64, device=d), algo=algo)
        assert out.numel() == 0
        assert p.solve_transpose(torch.zeros(0, dtype=torch.float64, device=d),
                                 algo=algo).numel() == 0
    p.reanalyze("auto")
    p.close()


def test_single_row_and_values_update():
    A = synth.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    with plan_for(A) as p:
        for algo in ALL_ALGOS:
            x = p.solve(torch.tensor([2.0], device=dev(), dtype=torch.float64), algo=algo)
            assert x.item() == 0.5, algo
        p.set_values(torch.tensor([8.0], device=dev(), dtype=torch.float64))
        for algo in ALL_ALGOS:
            x = p.solve(torch.tensor([2.0], device=dev(), dtype=torch.float64), algo=algo)
            assert x.item() == 0.25, algo


def test_values_change_without_reanalysis():
    """Sec. 1: ILU refactorisation keeps the pattern; solves see new values."""
    A = mat("general")
    with plan_for(A) as p:
        b = synth.uniform(A.n, 18)
        bt = torch.tensor(b, device=dev())
        p.solve(bt)
        p.vals.mul_(2.0)
        ref = oracle.solve(A.rowptr, A.colidx, 2.0 * A.vals, b)
        assert relerr(p.solve(bt), ref) <= TOL64


def test_autograd_sees_in_place_value_updates_with_copying_algorithms():
    """An optimizer step updates the values tensor in place; the autograd path
    must not solve from a stale level-ordered copy."""
    from paper_1710_04985_gb300 import sparse_triangular_solve
    A = mat("ilu_L")
    b = synth.uniform(A.n, 26)
    with plan_for(A) as p:
        v = p.vals
        bt = torch.tensor(b, device=dev())
        for algo in ("permuted", "blocked", "partitioned"):
            sparse_triangular_solve(p, v, bt, algo=algo)
            with torch.no_grad():
                v.mul_(0.5)
            x = sparse_triangular_solve(p, v, bt, algo=algo)
            ref = oracle.solve(A.rowptr, A.colidx, v.cpu().numpy(), b, unit=A.unit)
            assert relerr(x.detach(), ref) <= TOL64, algo


def test_c_abi_in_place_value_update_needs_refresh():
    """Through the C ABI: the default form (SPTRSV_ALGO_AUTO) is the
    partitioned one, which solves from a snapshot of the values.  Rewriting
    d_vals in place leaves the snapshot stale until sptrsv_refresh_values;
    after it the solve matches the oracle on the new values."""
    import ctypes

    from paper_1710_04985_gb300 import _lib
    lib = _lib.load()
    A = mat("general")
    b = synth.uniform(A.n, 61)
    with plan_for(A) as p:
        h = p._h
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        bt = torch.tensor(b, device=dev())
        x = torch.empty_like(bt)

        def solve_auto():
            assert lib.sptrsv_solve(h, ctypes.c_void_p(bt.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), 1, 1, _lib.ALGO_AUTO, s) == 0
            return x.clone()

        assert lib.sptrsv_set_default_algo(h, _lib.ALGO_SELF_PARTITIONED) == 0
        x0 = solve_auto()
        assert relerr(x0, oracle.solve(A.rowptr, A.colidx, A.vals, b)) <= TOL64
        p.vals.mul_(1.5)                                  # in place: same pointer
        assert torch.equal(solve_auto(), x0)              # the snapshot is stale
        assert lib.sptrsv_refresh_values(h, s) == 0
        ref = oracle.solve(A.rowptr, A.colidx, 1.5 * A.vals, b)
        assert relerr(solve_auto(), ref) <= TOL64


@pytest.mark.parametrize("algo", ["permuted", "partitioned"])
def test_level_ordered_copy_follows_value_updates(algo):
    """The level- and part-ordered copies are snapshots of the values:
    sptrsv_refresh_values (in-place change) and sptrsv_set_values (new array)
    bring them up to date, for the forward and the transposed copy."""
    A = mat("ilu_U")
    with plan_for(A) as p:
        b = synth.uniform(A.n, 24)
        bt = torch.tensor(b, device=dev())
        p.solve(bt, algo=algo)
        p.solve_transpose(bt, algo=algo)
        p.vals.mul_(2.0)
        p.refresh_values()
        ref = oracle.solve(A.rowptr, A.colidx, 2.0 * A.vals, b, upper=True)
        assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
        v3 = torch.tensor(3.0 * A.vals, device=dev())
        p.set_values(v3)
        ref = oracle.solve(A.rowptr, A.colidx, 3.0 * A.vals, b, upper=True)
        assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
        reft = oracle.solve_transpose(A.rowptr, A.colidx, 3.0 * A.vals, b, upper=True)
        assert relerr(p.solve_transpose(bt, algo=algo), reft) <= TOL64


@pytest.mark.parametrize("name", ["ilu_L", "ilu_U", "general", "general_upper", "bidiag",
                                  "bidiag_upper", "diag", "long_rows", "unit_nodiag",
                                  "lap3d_27pt", "lap2d_9pt_upper"])
def test_partitioned_part_sizes(name):
    """Parts of one row, ragged last parts, one part for the whole matrix and
    the automatic size; every lanes-per-row; a grid smaller than the parts.
    Each lane folds its entries in the order of the self-scheduled kernel,
    so the results are bitwise equal to it, and within 1e-12 of the oracle."""
    A = mat(name)
    b = synth.uniform(A.n, 27)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
    with plan_for(A) as p:
        bt = torch.tensor(b, device=dev())
        for lanes, block, grid in ((1, 128, 0), (4, 256, 0), (32, 1024, 5)):
            p.set_tuning(lanes, block, grid)
            p.set_partition(0)
            first = p.solve(bt)
            assert relerr(first, ref) <= TOL64
            for rows in (1, 33, 960, A.n, 0):
                for cl in (1, 2, 8):             # thread-block clusters of parts
                    p.set_partition(rows, cl)
                    assert torch.equal(p.solve(bt, algo="partitioned"), first), (lanes, rows, cl)
        assert p.status() == (0, -1)
        p.set_partition(1 << 30, 4)           # reduced to what fits shared memory
        assert 1000 <= p.partition < (1 << 30) and p.partition_shape[1] == 4
        assert relerr(p.solve(bt, algo="partitioned"), ref) <= TOL64
        from paper_1710_04985_gb300 import SptrsvError
        for bad in ((-1, 1), (0, 3), (0, 16)):
            with pytest.raises(SptrsvError):
                p.set_partition(*bad)


@pytest.mark.parametrize("cluster", [1, 4])
def test_partitioned_repeated_solves_and_graph_replays(cluster):
    """Every partitioned solve starts from a publication buffer and a ticket
    that the previous solve left behind.  A value or a ticket carried over
    would hand a dependent row the result of an earlier solve, or skip parts,
    so solves with a new right-hand side each time (both directions, grids
    smaller than the parts, and CUDA-graph replays of one captured solve)
    must each stay within 1e-12 of the oracle, and an unchanged right-hand
    side must give bitwise the same x."""
    A = mat("ilu_L")
    with plan_for(A) as p:
        p.set_partition(240, cluster)
        for lanes, block, grid in ((1, 128, 0), (1, 128, cluster), (4, 256, 0)):
            p.set_tuning(lanes, block, grid)
            first = None
            for k in range(5):
                b = synth.uniform(A.n, 300 + k)
                bt = torch.tensor(b, device=dev())
                ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
                assert relerr(p.solve(bt, algo="partitioned"), ref) <= TOL64, (lanes, grid, k)
                reft = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, b, upper=A.upper,
                                              unit=A.unit)
                assert relerr(p.solve_transpose(bt, algo="partitioned"), reft) <= TOL64
                if k == 0:
                    b0, first = bt, p.solve(bt, algo="partitioned")
            assert torch.equal(p.solve(b0, algo="partitioned"), first)
        assert p.status() == (0, -1)
        # graph replays of one captured solve, a new right-hand side each time
        p.set_tuning(1, 128, 0)
        bs = torch.zeros(A.n, dtype=torch.float64, device=dev())
        xs = torch.empty_like(bs)
        p.solve(bs, out=xs, algo="partitioned")
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            p.solve(bs, out=xs, algo="partitioned")
        for k in range(4):
            b = synth.uniform(A.n, 400 + k)
            bs.copy_(torch.tensor(b, device=dev()))
            g.replay()
            ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
            assert relerr(xs, ref) <= TOL64, k
        assert p.status() == (0, -1)


def _bad(n, rows, cols, vals, upper=False, unit=False):
    rows = np.asarray(rows)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return synth.CSR(n, rowptr, np.asarray(cols, np.int32), np.asarray(vals, float),
                     upper=upper, unit=unit)


@pytest.mark.parametrize("case,code,row", [
    ("unsorted", 2, 2), ("duplicate", 2, 1), ("upper_entry_in_lower", 2, 1),
    ("column_out_of_range", 2, 2), ("missing_diagonal", 3, 1), ("zero_diagonal", 3, 2),
    ("lower_entry_in_upper", 2, 1),
])
def test_structural_errors(case, code, row):
    from paper_1710_04985_gb300 import SptrsvError
    cases = {
        "unsorted": _bad(3, [0, 1, 1, 2, 2, 2], [0, 0, 1, 1, 0, 2], [1, 1, 1, 1, 1, 1]),
        "duplicate": _bad(3, [0, 1, 1, 1, 2], [0, 0, 0, 1, 2], [1, 1, 1, 1, 1]),
        "upper_entry_in_lower": _bad(3, [0, 1, 1, 2], [0, 1, 2, 2], [1, 1, 1, 1]),
        "column_out_of_range": _bad(3, [0, 1, 2, 2], [0, 1, 2, 9], [1, 1, 1, 1]),
        "missing_diagonal": _bad(3, [0, 1, 2], [0, 0, 2], [1, 1, 1]),
        "zero_diagonal": _bad(3, [0, 1, 2, 2], [0, 1, 1, 2], [1, 1, 1, 0.0]),
        "lower_entry_in_upper": _bad(3, [0, 1, 1, 2], [0, 0, 1, 2], [1, 1, 1, 1], upper=True),
    }
    with pytest.raises(SptrsvError) as ei:
        plan_for(cases[case])
    assert ei.value.status == code and ei.value.row == row


def test_bad_rowptr():
    from paper_1710_04985_gb300 import SptrsvError
    A = synth.CSR(3, np.array([0, 2, 1, 3], np.int32), np.array([0, 0, 1], np.int32),
                  np.ones(3))
    with pytest.raises(SptrsvError) as ei:
        plan_for(A)
    assert ei.value.status == 2


@pytest.mark.parametrize("algo", ["self", "tiled", "chains", "permuted", "column", "blocked",
                                  "partitioned"])
def test_timeout_is_reported_and_solve_finishes(algo):
    """A row that is never published: every row that depends on it gives up
    after the spin limit, records SPTRSV_ERR_TIMEOUT and publishes NaN; rows
    independent of it are still exact.  The GPU stays usable."""
    A = bidiagonal(2000)
    withheld = 300
    with plan_for(A) as p:
        p.set_spin_limit(1 << 14)
        p.withhold_row(withheld)
        b = synth.uniform(A.n, 19)
        x = p.solve(torch.tensor(b, device=dev()), algo=algo).cpu().numpy()
        st, row = p.status()
        assert st == 6 and row == withheld + 1
        ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
        assert relerr(x[:withheld], ref[:withheld]) <= TOL64
        assert np.all(np.isnan(x[withheld + 1:]))
        p.withhold_row(-1)
        assert relerr(p.solve(torch.tensor(b, device=dev()), algo=algo), ref) <= TOL64
        assert p.status() == (0, -1)


@pytest.mark.parametrize("cluster", [1, 2, 4])
@pytest.mark.parametrize("withheld", [300, 293])
def test_partitioned_timeout_in_part_and_across_the_cluster(cluster, withheld):
    """Bidiagonal chain, parts of 14 rows: row 300's dependent waits inside
    its part (shared memory), row 293's dependent (row 294, first row of the
    next part) waits in the previous block's shared memory when both parts
    belong to one cluster, else in L2.  Every such wait gives up after the
    spin limit with SPTRSV_ERR_TIMEOUT; the next solve is clean."""
    A = bidiagonal(2000)
    b = synth.uniform(A.n, 29)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with plan_for(A) as p:
        p.set_partition(14, cluster)
        p.set_tuning(1, 128, 0)
        p.set_spin_limit(1 << 14)
        p.withhold_row(withheld)
        x = p.solve(torch.tensor(b, device=dev()), algo="partitioned").cpu().numpy()
        assert p.status() == (6, withheld + 1)
        assert relerr(x[:withheld], ref[:withheld]) <= TOL64
        assert np.all(np.isnan(x[withheld + 1:]))
        p.withhold_row(-1)
        assert relerr(p.solve(torch.tensor(b, device=dev()), algo="partitioned"), ref) <= TOL64
        assert p.status() == (0, -1)


# ---------------------------------------------------------------- gradient / residual

@pytest.mark.parametrize("name", ["general", "ilu_L", "ilu_U", "unit_nodiag"])
def test_grad_vals_matches_oracle(name):
    A = mat(name)
    for k in (1, 3):
        y = synth.uniform((A.n, k), 20)
        x = synth.uniform((A.n, k), 21)
        ref = oracle.grad_vals(A.rowptr, A.colidx, y, x, unit=A.unit)
        with plan_for(A) as p:
            g = p.grad_vals(torch.tensor(y, device=dev()), torch.tensor(x, device=dev()))
            assert relerr(g, ref) <= 1e-14


@pytest.mark.parametrize("name", ["general", "ilu_L", "unit_nodiag", "general_upper"])
def test_residual_matches_oracle(name):
    """r = b - A x in FP64; a unit diagonal counts as 1 whether it is stored
    (ILU L factor) or not."""
    A = mat(name)
    b = synth.uniform((A.n, 2), 22)
    x = synth.uniform((A.n, 2), 23)
    ref = oracle.residual(A.rowptr, A.colidx, A.vals, b, x, unit=A.unit)
    with plan_for(A) as p:
        r = p.residual(torch.tensor(b, device=dev()), torch.tensor(x, device=dev()))
        assert relerr(r, ref) <= 1e-14


@pytest.mark.parametrize("transpose", [False, True])
def test_autograd_against_oracle_and_finite_differences(transpose):
    from paper_1710_04985_gb300 import sparse_triangular_solve
    A = mat("general")
    b = synth.uniform(A.n, 24)
    t = synth.uniform(A.n, 25)
    with plan_for(A) as p:
        v = torch.tensor(A.vals, device=dev()).requires_grad_(True)
        bb = torch.tensor(b, device=dev()).requires_grad_(True)
        tt = torch.tensor(t, device=dev())
        x = sparse_triangular_solve(p, v, bb, transpose=transpose)
        loss = 0.5 * ((x - tt) ** 2).sum()
        loss.backward()
        if transpose:
            xr = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, b)
            yr = oracle.solve(A.rowptr, A.colidx, A.vals, xr - t)
            gr = oracle.grad_vals(A.rowptr, A.colidx, xr, yr)
        else:
            xr = oracle.solve(A.rowptr, A.colidx, A.vals, b)
            yr = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, xr - t)
            gr = oracle.grad_vals(A.rowptr, A.colidx, yr, xr)
        assert relerr(bb.grad, yr) <= TOL64
        assert relerr(v.grad, gr) <= TOL64
        # central differences through the GPU solve
        rng = np.random.default_rng(26)

        def L(vals, bvec):
            with torch.no_grad():
                xx = sparse_triangular_solve(p, vals, bvec, transpose=transpose)
                return 0.5 * float(((xx - tt) ** 2).sum())

        v0 = v.detach().clone()
        b0 = bb.detach().clone()
        for q in rng.choice(A.nnz, 8, replace=False):
            h = 1e-5 * max(1.0, abs(A.vals[q]))
            vp, vm = v0.clone(), v0.clone()
            vp[q] += h
            vm[q] -= h
            fd = (L(vp, b0) - L(vm, b0)) / (2 * h)
            an = float(v.grad[q])
            assert abs(fd - an) <= 1e-4 * max(1.0, abs(an))
        for q in rng.choice(A.n, 8, replace=False):
            h = 1e-5
            bp, bm = b0.clone(), b0.clone()
            bp[q] += h
            bm[q] -= h
            fd = (L(v0, bp) - L(v0, bm)) / (2 * h)
            an = float(bb.grad[q])
            assert abs(fd - an) <= 1e-4 * max(1.0, abs(an))


# ---------------------------------------------------------------- precision

@pytest.mark.parametrize("name", ["general", "ilu_L", "ilu_U", "long_rows"])
@pytest.mark.parametrize("k", [1, 8])
@pytest.mark.parametrize("algo", ["self", "partitioned", "permuted", "blocked", "chains",
                                  "level"])
def test_fp32_with_fp64_refinement(name, k, algo):
    """The FP32 solves run the plan's default form: the in-place and copying
    forms add each correction into x as they publish it, the others through
    an update pass; every way reaches the FP64 oracle within 1e-12."""
    A = mat(name)
    b = synth.uniform((A.n, k) if k > 1 else A.n, 27)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
    with plan_for(A) as p:
        p.best_algo = algo
        p.set_partition(1024, 2)
        x, iters, rel = p.solve_refined(torch.tensor(b, device=dev()))
        err = relerr(x, ref)
        assert err <= TOL64, (err, iters, rel)
        assert 1 <= iters <= 10
        assert p.status() == (0, -1)
        if algo == "partitioned" and k == 1:
            # the FP32 copy follows value updates (refresh), like the FP64 one
            v2 = torch.tensor(A.vals * 1.25, device=dev())
            p.set_values(v2)
            ref2 = oracle.solve(A.rowptr, A.colidx, A.vals * 1.25, b, upper=A.upper,
                                unit=A.unit)
            x2, _, _ = p.solve_refined(torch.tensor(b, device=dev()))
            assert relerr(x2, ref2) <= TOL64


@pytest.mark.parametrize("name", ["general", "ilu_L", "ilu_U", "long_rows", "general_upper",
                                  "unit_nodiag"])
def test_one_pass_refinement_steps_and_passes(name):
    """One right-hand side in the one-pass form: every refinement step runs in
    one self-scheduled sweep.  Its result meets the FP64 oracle like the
    staged form's; with tol = 0 the solve keeps going pass after pass (later
    passes start from the current x) until max_iter corrections are spent;
    max_iter = 1 stops after the first pass's single correction."""
    A = mat(name)
    b = synth.uniform(A.n, 71)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
    with plan_for(A) as p:
        assert p.refine_mode == "staged"            # the default
        p.refine_mode = "one_pass"
        assert p.refine_mode == "one_pass"
        bt = torch.tensor(b, device=dev())
        for lanes in (1, 4, 32):
            p.set_tuning(lanes, 256, 0)
            x, iters, rel = p.solve_refined(bt)
            assert relerr(x, ref) <= TOL64, (lanes, iters, rel)
            assert 1 <= iters <= 10 and rel <= 8 * 2.0 ** -52
        x, iters, rel = p.solve_refined(bt, max_iter=7, tol=0.0)
        assert iters == 7 and relerr(x, ref) <= TOL64
        x, iters, rel = p.solve_refined(bt, max_iter=1)
        assert iters == 1 and relerr(x, ref) <= 1e-9
        p.refine_mode = "staged"
        xs, its, rels = p.solve_refined(bt)
        assert relerr(xs, ref) <= TOL64
        from paper_1710_04985_gb300 import autotune
        res = autotune.tune_refine(p, bt)
        assert p.refine_mode == res["mode"] and set(res["ms"]) == {"staged", "one_pass"}
        assert relerr(p.solve_refined(bt)[0], ref) <= TOL64
        assert p.status() == (0, -1)


# ---------------------------------------------------------------- batching

def test_batched_block_diagonal_graph():
    from paper_1710_04985_gb300 import BatchedTriangularSolve
    mats = synth.batch_general(24, seed=31, nmin=1000, nmax=8000)
    systems = [(m.rowptr, m.colidx, m.vals) for m in mats]
    bs = BatchedTriangularSolve(systems, tune=True)
    assert bs.tuning["best"][0] in (1, 2, 4, 8, 16, 32)
    bvecs = [synth.uniform(m.n, 100 + s) for s, m in enumerate(mats)]
    x = bs.solve(torch.tensor(np.concatenate(bvecs), device=dev())).cpu().numpy()
    lev = bs.plan.levels()["lev"].cpu().numpy()
    off = bs.offsets
    for s, m in enumerate(mats):
        ref = oracle.solve(m.rowptr, m.colidx, m.vals, bvecs[s])
        assert relerr(x[off[s]:off[s + 1]], ref) <= TOL64
        lref, _ = oracle.levels(m.rowptr, m.colidx)
        assert np.array_equal(lev[off[s]:off[s + 1]], lref)
    # replay with new right-hand sides
    b2 = [synth.uniform(m.n, 200 + s) for s, m in enumerate(mats)]
    x2 = bs.solve(torch.tensor(np.concatenate(b2), device=dev())).cpu().numpy()
    for s in (0, len(mats) - 1):
        m = mats[s]
        ref = oracle.solve(m.rowptr, m.colidx, m.vals, b2[s])
        assert relerr(x2[off[s]:off[s + 1]], ref) <= TOL64


def test_autotuner_keeps_results_exact():
    from paper_1710_04985_gb300 import autotune
    A = mat("ilu_L")
    b = synth.uniform(A.n, 32)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, unit=True)
    with plan_for(A) as p:
        bt = torch.tensor(b, device=dev())
        res = autotune.tune(p, bt, use_cache=False, blocks=(128, 256))
        assert len(res["table"]) == 6 + 2 * 4 - 1
        assert p.tuning["lanes_per_row"] == res["best"][0]
        assert p.tuning["max_blocks"] == res["best"][2]
        assert relerr(p.solve(bt), ref) <= TOL64


def test_autotuner_picks_an_algorithm_and_stays_exact():
    from paper_1710_04985_gb300 import autotune
    A = mat("general")
    b = synth.uniform(A.n, 33)
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with plan_for(A) as p:
        bt = torch.tensor(b, device=dev())
        res = autotune.tune_algos(p, bt, use_cache=False, lanes=(2, 8), blocks=(256,),
                                  grids=(0, 2), tiles=(512, 2048))
        assert res["algo"] in ("self", "permuted", "blocked", "partitioned", "tiled", "chains")
        assert p.best_algo == res["algo"]
        assert relerr(p.solve(bt, algo="auto"), ref) <= TOL64
