"""Full-size parity: the workloads at their real sizes, in the launch
configuration the benchmark times (autotuned self-scheduled solve), compared
element by element with the oracle (its sequential solves finish in well
under a second at these sizes)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL32, TOL64, assert_levels_equal, dev, plan_for, relerr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def w1(cuda_device):
    return synth.workload1()


@pytest.fixture(scope="module")
def w2(cuda_device):
    return synth.workload2()


def bench_plan(A, b, dtype=torch.float64):
    """The plan as the benchmark builds it: analysed, then autotuned over the
    self-scheduled forms (in place, level-ordered copy, blocked, partitioned,
    tiled, chained); each form keeps its own tuned launch shape."""
    from paper_1710_04985_gb300 import autotune
    p = plan_for(A, dtype)
    autotune.tune_algos(p, torch.tensor(b, device=dev(), dtype=dtype))
    return p


def test_workload1_ilu_factors_forward_and_backward(w1):
    L, U, xt, bL, bU = w1
    assert (L.n, L.nnz, U.nnz) == (2097152, 8339456, 8339456)
    for A, b in ((L, bL), (U, bU)):
        ref = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
        with bench_plan(A, b) as p:
            assert_levels_equal(p.levels(), A)
            assert p.levels()["nlev"] == 382
            bt = torch.tensor(b, device=dev())
            for algo in ("auto", "self", "permuted", "partitioned", "tiled", "level"):
                assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
            assert relerr(ref, xt) <= 1e-10           # manufactured solution recovered
            assert p.status() == (0, -1)


def test_workload1_solve_pair(w1):
    """The benchmark step: y = U^{-1} (L^{-1} b) (eq. (3))."""
    L, U, xt, _, _ = w1
    b = synth.times_vector(L, synth.times_vector(U, xt))
    with bench_plan(L, b) as pl, bench_plan(U, b) as pu:
        y = pu.solve(pl.solve(torch.tensor(b, device=dev()), algo="auto"), algo="auto")
        assert relerr(y, xt) <= 1e-10
        ref = oracle.solve(U.rowptr, U.colidx, U.vals,
                           oracle.solve(L.rowptr, L.colidx, L.vals, b, unit=True), upper=True)
        assert relerr(y, ref) <= TOL64


@pytest.mark.parametrize("k", [8, 32])
def test_workload3_multi_rhs_on_ilu_L(w1, k):
    L = w1[0]
    b = synth.uniform((L.n, k), 3000 + k)
    ref = oracle.solve(L.rowptr, L.colidx, L.vals, b, unit=True)
    with plan_for(L) as p:
        assert relerr(p.solve(torch.tensor(b, device=dev())), ref) <= TOL64


def test_workload3_refinement_on_ilu_L(w1):
    L = w1[0]
    b = synth.uniform((L.n, 8), 3100)
    ref = oracle.solve(L.rowptr, L.colidx, L.vals, b, unit=True)
    with plan_for(L) as p:
        x, iters, rel = p.solve_refined(torch.tensor(b, device=dev()))
        assert relerr(x, ref) <= TOL64 and iters <= 10


def test_workload2_general_fp64_fp32(w2):
    A, xt, b = w2
    assert A.n == 1_000_000
    ref = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    with bench_plan(A, b) as p:
        assert_levels_equal(p.levels(), A)
        bt = torch.tensor(b, device=dev())
        for algo in ("auto", "self", "permuted", "tiled", "level"):
            assert relerr(p.solve(bt, algo=algo), ref) <= TOL64
    with bench_plan(A, b, torch.float32) as p32:
        x32 = p32.solve(torch.tensor(b, device=dev(), dtype=torch.float32), algo="auto")
        assert relerr(x32.double(), ref) <= TOL32
    with plan_for(A) as p:
        x, iters, rel = p.solve_refined(torch.tensor(b, device=dev()))
        assert relerr(x, ref) <= TOL64


@pytest.mark.parametrize("dims,pts", [((1024, 1024), 9), ((128, 128, 128), 27),
                                      ((64, 16384), 5), ((32, 32, 2048), 7)])
def test_table2_stencil_pair(dims, pts):
    """Sec. 5.1 at full size: the solve pair of eq. (3) on Table 2 grids, in
    the launch configuration the sweep times (autotuned), against the oracle
    and the manufactured solution; levels bit-exact."""
    L, U = synth.laplacian_triangles(dims, pts)
    xt = synth.uniform(L.n, synth.SEED_BASE + 10 + pts)
    b = synth.times_vector(L, synth.times_vector(U, xt))
    c = oracle.solve(L.rowptr, L.colidx, L.vals, b)
    ref = oracle.solve(U.rowptr, U.colidx, U.vals, c, upper=True)
    assert relerr(ref, xt) <= 1e-10
    with bench_plan(L, b) as pl:
        assert_levels_equal(pl.levels(), L)
        y = pl.solve(torch.tensor(b, device=dev()), algo="auto")
        assert relerr(y, c) <= TOL64
        with bench_plan(U, c) as pu:
            assert_levels_equal(pu.levels(), U)
            for algo in ("auto", "self", "permuted"):
                assert relerr(pu.solve(y, algo=algo), ref) <= TOL64


def test_workload4_gradient(w2):
    """loss = 0.5 ||A^{-1} b - t||^2 on the n = 10^6 general matrix: autograd
    against the oracle gradient and central differences on 64 coordinates."""
    from paper_1710_04985_gb300 import sparse_triangular_solve
    A = w2[0]
    b = synth.uniform(A.n, synth.SEED_BASE + 4)
    t = synth.uniform(A.n, synth.SEED_BASE + 4 + 1)
    xr = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    yr = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, xr - t)
    gr = oracle.grad_vals(A.rowptr, A.colidx, yr, xr)
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        with plan_for(A, dtype) as p:
            v = torch.tensor(A.vals, device=dev(), dtype=dtype).requires_grad_(True)
            bb = torch.tensor(b, device=dev(), dtype=dtype).requires_grad_(True)
            tt = torch.tensor(t, device=dev(), dtype=dtype)
            x = sparse_triangular_solve(p, v, bb)
            (0.5 * ((x - tt) ** 2).sum()).backward()
            assert relerr(bb.grad.double(), yr) <= tol
            assert relerr(v.grad.double(), gr) <= tol
            if dtype != torch.float64:
                continue
            rng = np.random.default_rng(synth.SEED_BASE + 4)
            v0, b0 = v.detach().clone(), bb.detach().clone()

            def loss(vals, bvec):
                with torch.no_grad():
                    xx = sparse_triangular_solve(p, vals, bvec)
                    return 0.5 * float(((xx - tt) ** 2).sum())

            for q in rng.choice(A.nnz, 32, replace=False):
                h = 1e-5 * max(1.0, abs(A.vals[q]))
                vp, vm = v0.clone(), v0.clone()
                vp[q] += h
                vm[q] -= h
                fd = (loss(vp, b0) - loss(vm, b0)) / (2 * h)
                an = float(v.grad[q])
                assert abs(fd - an) <= 1e-4 * max(1.0, abs(an)), (q, fd, an)
            for q in rng.choice(A.n, 32, replace=False):
                h = 1e-5
                bp, bm = b0.clone(), b0.clone()
                bp[q] += h
                bm[q] -= h
                fd = (loss(v0, bp) - loss(v0, bm)) / (2 * h)
                an = float(bb.grad[q])
                assert abs(fd - an) <= 1e-4 * max(1.0, abs(an)), (q, fd, an)


def test_workload3_batch_of_512_systems(cuda_device):
    """512 independent general systems, n log-uniform in [1k, 64k], solved by
    one graph-replayed launch of the autotuned plan; every system checked
    against its own oracle solve, and the block-diagonal levels against the
    per-system levels.  Then the same batch on the partitioned form (the
    system boundaries found by the plan: one independent block per system)
    and by FP32 solves with FP64 refinement, both against the oracle."""
    from paper_1710_04985_gb300 import BatchedTriangularSolve
    mats = synth.batch_general_parallel(512, synth.SEED_BASE + 3)
    bs = BatchedTriangularSolve([(m.rowptr, m.colidx, m.vals) for m in mats], tune=True)
    bvec = [synth.uniform(m.n, 7000 + s) for s, m in enumerate(mats)]
    bt = torch.tensor(np.concatenate(bvec), device=dev())
    x = bs.solve(bt).cpu().numpy()
    lev = bs.plan.levels()["lev"].cpu().numpy()
    off = bs.offsets
    refs = [oracle.solve(m.rowptr, m.colidx, m.vals, bvec[s]) for s, m in enumerate(mats)]

    def worst(xs):
        return max(relerr(xs[off[s]:off[s + 1]], refs[s]) for s in range(len(mats)))

    for s, m in enumerate(mats):
        lref, _ = oracle.levels(m.rowptr, m.colidx)
        assert np.array_equal(lev[off[s]:off[s + 1]], lref)
    assert worst(x) <= TOL64
    xp = bs.plan.solve(bt, algo="partitioned").cpu().numpy()
    assert worst(xp) <= TOL64
    assert bs.plan.partition_info()["nblocks"] == 512
    xr, iters, rel = bs.solve_refined(bt)
    assert 1 <= iters <= 10
    assert worst(xr.cpu().numpy()) <= TOL64
    assert bs.plan.status() == (0, -1)
