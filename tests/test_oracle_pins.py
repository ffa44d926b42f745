"""Pins for the CPU oracle: checks against facts fixed by the paper or by the
mathematics, never against the oracle itself.

* dense triangular solves (scipy/LAPACK) on tiny random patterns
* manufactured solutions (x chosen, b = A x through scipy)
* closed forms for levels (Sec. 4.1: nlev = nx+ny-1 and nx+ny+nz-2; derived
  here for the 9- and 27-point stencils of Sec. 5.1)
* the worked example of Fig. 1 (golden fixture)
* brute-force longest paths on tiny random DAGs
* level invariants (one level per row, deps strictly lower, tightness)
* adjoint identity and central finite differences for the gradient
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_triangle(n, density, seed, upper=False, unit=False, store_diag=True):
    """Tiny random triangular CSR with a well-conditioned diagonal."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        cand = np.arange(i + 1, n) if upper else np.arange(0, i)
        pick = cand[rng.random(cand.size) < density]
        entries = list(pick)
        if store_diag:
            entries.append(i)
        for j in sorted(entries):
            rows.append(i)
            cols.append(j)
            vals.append(rng.uniform(-1, 1) if j != i else
                        rng.choice([-1, 1]) * rng.uniform(2.0, 4.0))
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return synth.CSR(n, rowptr, cols.astype(np.int32), np.array(vals), upper=upper, unit=unit)


def dense(A):
    M = A.scipy().toarray()
    if A.unit:
        np.fill_diagonal(M, 1.0)
    return M


# ---------------------------------------------------------------- solves

@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("unit", [False, True])
def test_solve_matches_dense_lapack(n, upper, unit):
    A = random_triangle(n, 0.3, seed=n * 7 + upper * 3 + unit, upper=upper, unit=unit,
                        store_diag=not unit or n % 2 == 0)
    rng = np.random.default_rng(n)
    b = rng.uniform(-1, 1, (n, 3))
    want = sla.solve_triangular(dense(A), b, lower=not upper, unit_diagonal=unit)
    got = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=upper, unit=unit)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    got1 = oracle.solve(A.rowptr, A.colidx, A.vals, b[:, 1], upper=upper, unit=unit)
    np.testing.assert_allclose(got1, want[:, 1], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n", [1, 5, 40])
@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("unit", [False, True])
def test_solve_transpose_matches_dense_lapack(n, upper, unit):
    A = random_triangle(n, 0.35, seed=100 + n, upper=upper, unit=unit)
    g = np.random.default_rng(n + 1).uniform(-1, 1, (n, 2))
    want = sla.solve_triangular(dense(A).T, g, lower=upper, unit_diagonal=unit)
    got = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, g, upper=upper, unit=unit)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_manufactured_solution_general():
    A = synth.general_lower(5000, seed=3)
    xt = synth.uniform(A.n, 4)
    b = synth.times_vector(A, xt)
    x = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    assert np.max(np.abs(x - xt)) <= 1e-13


def test_manufactured_solution_workload0():
    A, xt, b = synth.workload0()
    assert (A.n, A.nnz) == (4096, 12160)
    x = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    assert np.max(np.abs(x - xt)) / np.max(np.abs(xt)) <= 1e-13


def test_manufactured_solution_ilu_factors_small():
    L, U = synth.lap3d_7pt_ilu0(9, 7, 5)
    xt = synth.uniform(L.n, 5)
    for A in (L, U):
        b = synth.times_vector(A, xt)
        x = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=A.upper, unit=A.unit)
        assert np.max(np.abs(x - xt)) <= 1e-13


def test_diagonal_matrix_special_case():
    n = 50
    d = np.linspace(1.0, 3.0, n)
    rowptr = np.arange(n + 1, dtype=np.int32)
    colidx = np.arange(n, dtype=np.int32)
    b = np.linspace(-1, 1, n)
    np.testing.assert_allclose(oracle.solve(rowptr, colidx, d, b), b / d, rtol=1e-15)
    lev, nlev = oracle.levels(rowptr, colidx)
    assert nlev == 1 and not lev.any()


def test_bidiagonal_is_fully_sequential():
    """Sec. 4.1: the worst case nlev = n."""
    n = 300
    rows = np.repeat(np.arange(n), 2)[1:]
    cols = np.sort(np.concatenate([np.arange(n), np.arange(n - 1)]))
    rowptr = np.concatenate([[0], np.cumsum(np.minimum(np.arange(1, n + 1), 2))]).astype(np.int32)
    vals = np.where(np.repeat(np.arange(n), np.diff(rowptr)) == cols, 2.0, -1.0)
    A = synth.CSR(n, rowptr, cols.astype(np.int32), vals)
    lev, nlev = oracle.levels(A.rowptr, A.colidx)
    assert nlev == n and np.array_equal(lev, np.arange(n))
    b = np.ones(n)
    want = sla.solve_triangular(dense(A), b, lower=True)
    np.testing.assert_allclose(oracle.solve(A.rowptr, A.colidx, A.vals, b), want, rtol=1e-12)
    assert rows.size == A.nnz


# ---------------------------------------------------------------- levels

@pytest.mark.parametrize("nx,ny", [(64, 64), (5, 5), (1, 9), (13, 4)])
def test_levels_closed_form_2d(nx, ny):
    """Sec. 4.1: nlev = nx + ny - 1; the level of grid point (x, y) is x + y
    in the lower sweep and (nx-1-x) + (ny-1-y) in the upper sweep."""
    A = synth.lap2d_5pt_lower(nx, ny)
    lev, nlev = oracle.levels(A.rowptr, A.colidx)
    x, y = np.arange(A.n) % nx, np.arange(A.n) // nx
    assert nlev == nx + ny - 1
    assert np.array_equal(lev, x + y)
    U = synth.lap2d_5pt_upper(nx, ny)
    levu, nlevu = oracle.levels(U.rowptr, U.colidx, upper=True)
    assert nlevu == nx + ny - 1
    assert np.array_equal(levu, (nx - 1 - x) + (ny - 1 - y))


@pytest.mark.parametrize("dims", [(6, 5, 4), (16, 12, 10), (128, 128, 128)])
def test_levels_closed_form_3d(dims):
    """Sec. 4.1: nlev = nx + ny + nz - 2 for the 7-point operator."""
    nx, ny, nz = dims
    L, U = synth.lap3d_7pt_ilu0(nx, ny, nz)
    i = np.arange(L.n)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    lev, nlev = oracle.levels(L.rowptr, L.colidx)
    assert nlev == nx + ny + nz - 2
    assert np.array_equal(lev, x + y + z)
    levu, nlevu = oracle.levels(U.rowptr, U.colidx, upper=True)
    assert nlevu == nx + ny + nz - 2
    assert np.array_equal(levu, (nx - 1 - x) + (ny - 1 - y) + (nz - 1 - z))


@pytest.mark.parametrize("nx,ny", [(2, 2), (7, 5), (5, 9), (64, 16)])
def test_levels_closed_form_9pt(nx, ny):
    """9-point stencil (Sec. 5.1, Table 2), nx >= 2: the dependency on
    (x+1, y-1) makes each grid line two levels deep, so lev = x + 2y and
    nlev = nx + 2 ny - 2 (the upper sweep is the point reflection)."""
    L, U = synth.laplacian_triangles((nx, ny), 9)
    x, y = np.arange(L.n) % nx, np.arange(L.n) // nx
    lev, nlev = oracle.levels(L.rowptr, L.colidx)
    assert nlev == nx + 2 * ny - 2
    assert np.array_equal(lev, x + 2 * y)
    levu, nlevu = oracle.levels(U.rowptr, U.colidx, upper=True)
    assert nlevu == nlev
    assert np.array_equal(levu, (nx - 1 - x) + 2 * (ny - 1 - y))


@pytest.mark.parametrize("dims", [(2, 2, 2), (6, 5, 4), (4, 7, 9)])
def test_levels_closed_form_27pt(dims):
    """27-point stencil, nx, ny >= 2: the dependencies on (x+1, y-1, z) and
    (x+1, y+1, z-1) give lev = x + 2y + 4z, nlev = nx + 2 ny + 4 nz - 6."""
    nx, ny, nz = dims
    L, U = synth.laplacian_triangles(dims, 27)
    i = np.arange(L.n)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    lev, nlev = oracle.levels(L.rowptr, L.colidx)
    assert nlev == nx + 2 * ny + 4 * nz - 6
    assert np.array_equal(lev, x + 2 * y + 4 * z)
    levu, nlevu = oracle.levels(U.rowptr, U.colidx, upper=True)
    assert nlevu == nlev
    assert np.array_equal(levu, (nx - 1 - x) + 2 * (ny - 1 - y) + 4 * (nz - 1 - z))


def test_levels_closed_form_table2_grids():
    """Level counts of the Table 2 grids follow the closed forms (and grow
    with the aspect ratios of eq. (5), as Sec. 5.1 says)."""
    for nx, ny in synth.TABLE2_GRIDS_2D[:2]:
        for pts, want in ((5, nx + ny - 1), (9, nx + 2 * ny - 2)):
            L, _ = synth.laplacian_triangles((nx, ny), pts)
            assert oracle.levels(L.rowptr, L.colidx)[1] == want
    nx, ny, nz = synth.TABLE2_GRIDS_3D[-1]
    L, _ = synth.laplacian_triangles((nx, ny, nz), 7)
    assert oracle.levels(L.rowptr, L.colidx)[1] == nx + ny + nz - 2


def read_golden_fig1():
    out = {"levels": {}, "deps": {}}
    with open(os.path.join(GOLDEN, "fig1_5x5_levels.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            head, _, tail = line.partition(":")
            words = head.split()
            if words[0] == "grid":
                out["grid"] = (int(words[1]), int(words[2]))
            elif words[0] == "nlev":
                out["nlev"] = int(words[1])
            elif words[0] == "level":
                out["levels"][int(words[1])] = [int(t) for t in tail.split()]
            elif words[0] == "deps":
                out["deps"][int(words[1])] = [int(t) for t in tail.split()]
    return out


def test_fig1_worked_example():
    g = read_golden_fig1()
    nx, ny = g["grid"]
    A = synth.lap2d_5pt_lower(nx, ny)
    lev, nlev = oracle.levels(A.rowptr, A.colidx)
    assert nlev == g["nlev"]
    ilev, jlev = oracle.level_sets(lev, nlev)
    for paper_level, nodes in g["levels"].items():
        m = paper_level - 1                       # 0-based level
        assert sorted((jlev[ilev[m]:ilev[m + 1]] + 1).tolist()) == nodes
    for node, deps in g["deps"].items():
        i = node - 1
        row = A.colidx[A.rowptr[i]:A.rowptr[i + 1]]
        assert sorted((row[row != i] + 1).tolist()) == deps


def longest_path_levels(n, deps):
    """Brute force: level = length of the longest dependency chain ending at
    the node, by memoised depth-first search."""
    memo = {}

    def depth(v):
        if v in memo:
            return memo[v]
        best = 0
        for u in deps[v]:
            best = max(best, depth(u) + 1)
        memo[v] = best
        return best

    return np.array([depth(v) for v in range(n)], dtype=np.int64)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("upper", [False, True])
def test_levels_brute_force(seed, upper):
    n = 40
    A = random_triangle(n, 0.15, seed=seed, upper=upper)
    deps = [[j for j in A.colidx[A.rowptr[i]:A.rowptr[i + 1]] if j != i] for i in range(n)]
    lev, nlev = oracle.levels(A.rowptr, A.colidx, upper=upper)
    want = longest_path_levels(n, deps)
    assert np.array_equal(lev, want) and nlev == want.max() + 1
    # transposed system: i depends on j when A_ji != 0
    tdeps = [[] for _ in range(n)]
    for j in range(n):
        for i in A.colidx[A.rowptr[j]:A.rowptr[j + 1]]:
            if i != j:
                tdeps[i].append(j)
    tlev, tnlev = oracle.levels_transpose(A.rowptr, A.colidx, upper=upper)
    twant = longest_path_levels(n, tdeps)
    assert np.array_equal(tlev, twant) and tnlev == twant.max() + 1


def test_levels_transpose_equal_levels_of_explicit_transpose():
    """Column-wise loop on A (Sec. 4.1) = row-wise loop on scipy's A^T."""
    A = synth.general_lower(3000, seed=11)
    T = A.scipy().T.tocsr()
    T.sort_indices()
    want, wn = oracle.levels(T.indptr.astype(np.int32), T.indices.astype(np.int32), upper=True)
    got, gn = oracle.levels_transpose(A.rowptr, A.colidx, upper=False)
    assert gn == wn and np.array_equal(got, want)


def check_level_invariants(A, lev, nlev):
    n = A.n
    rows = A.row_of_entries()
    off = A.colidx != rows
    assert lev.min() >= 0 and lev.max() == nlev - 1
    # every dependency sits on a strictly lower level
    assert np.all(lev[A.colidx[off]] < lev[rows[off]])
    # tightness: a row with lev > 0 has a dependency exactly one level down
    best = np.full(n, -1)
    np.maximum.at(best, rows[off], lev[A.colidx[off]])
    assert np.array_equal(lev, best + 1)


def test_level_invariants_general():
    A = synth.general_lower(20000, seed=21)
    lev, nlev = oracle.levels(A.rowptr, A.colidx)
    check_level_invariants(A, lev, nlev)


def test_level_sets_are_a_stable_counting_sort():
    A = synth.general_lower(20000, seed=22)
    lev, nlev = oracle.levels(A.rowptr, A.colidx)
    ilev, jlev = oracle.level_sets(lev, nlev)
    assert ilev[0] == 0 and ilev[-1] == A.n and np.all(np.diff(ilev) > 0)
    assert np.array_equal(np.sort(jlev), np.arange(A.n))            # a permutation
    assert np.array_equal(jlev, np.argsort(lev, kind="stable"))      # numpy's stable sort
    assert np.array_equal(np.diff(ilev), np.bincount(lev, minlength=nlev))
    for m in (0, nlev // 2, nlev - 1):                               # partition by level
        assert np.all(lev[jlev[ilev[m]:ilev[m + 1]]] == m)


# ---------------------------------------------------------------- adjoint / gradient

def test_adjoint_identity():
    """<A^{-1} b, g> = <b, A^{-T} g>."""
    A = synth.general_lower(4000, seed=31)
    b = synth.uniform(A.n, 32)
    g = synth.uniform(A.n, 33)
    x = oracle.solve(A.rowptr, A.colidx, A.vals, b)
    y = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, g)
    assert abs(x @ g - b @ y) <= 1e-12 * max(1.0, abs(x @ g))


@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("unit", [False, True])
def test_gradient_finite_differences(upper, unit):
    """loss = 0.5 ||A^{-1} b - t||^2: oracle gradient vs central differences."""
    A = random_triangle(30, 0.3, seed=41 + upper + 2 * unit, upper=upper, unit=unit)
    rng = np.random.default_rng(7)
    b = rng.uniform(-1, 1, A.n)
    t = rng.uniform(-1, 1, A.n)

    def loss(vals, bb):
        x = oracle.solve(A.rowptr, A.colidx, vals, bb, upper=upper, unit=unit)
        return 0.5 * np.sum((x - t) ** 2)

    x = oracle.solve(A.rowptr, A.colidx, A.vals, b, upper=upper, unit=unit)
    y = oracle.solve_transpose(A.rowptr, A.colidx, A.vals, x - t, upper=upper, unit=unit)
    gv = oracle.grad_vals(A.rowptr, A.colidx, y, x, unit=unit)
    h = 1e-6
    for p in rng.choice(A.nnz, 12, replace=False):
        v1, v2 = A.vals.copy(), A.vals.copy()
        v1[p] += h
        v2[p] -= h
        fd = (loss(v1, b) - loss(v2, b)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-6 * max(1.0, abs(gv[p]))
    for q in rng.choice(A.n, 6, replace=False):
        b1, b2 = b.copy(), b.copy()
        b1[q] += h
        b2[q] -= h
        fd = (loss(A.vals, b1) - loss(A.vals, b2)) / (2 * h)
        assert abs(fd - y[q]) <= 1e-6 * max(1.0, abs(y[q]))


def test_gradient_matches_dense_outer_product():
    A = random_triangle(25, 0.4, seed=51)
    rng = np.random.default_rng(8)
    y = rng.uniform(-1, 1, (A.n, 2))
    x = rng.uniform(-1, 1, (A.n, 2))
    G = -(y @ x.T)
    rows = A.row_of_entries()
    np.testing.assert_allclose(oracle.grad_vals(A.rowptr, A.colidx, y, x), G[rows, A.colidx],
                               rtol=1e-14, atol=1e-14)


def test_residual_matches_scipy():
    A = synth.general_lower(3000, seed=61)
    rng = np.random.default_rng(9)
    b = rng.uniform(-1, 1, (A.n, 3))
    x = rng.uniform(-1, 1, (A.n, 3))
    want = b - sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n)) @ x
    np.testing.assert_allclose(oracle.residual(A.rowptr, A.colidx, A.vals, b, x), want,
                               rtol=1e-12, atol=1e-12)
    L, _ = synth.lap3d_7pt_ilu0(5, 4, 3)         # unit diagonal stored as 1.0
    L2 = L.with_vals(np.where(L.row_of_entries() == L.colidx, 7.0, L.vals))
    xx = rng.uniform(-1, 1, L.n)
    bb = synth.times_vector(L, xx)
    r = oracle.residual(L2.rowptr, L2.colidx, L2.vals, bb, xx, unit=True)
    assert np.max(np.abs(r)) <= 1e-14
    # a unit diagonal that is not stored still counts as 1 (the unit flag's
    # reading): r = b - (strict lower part + I) x
    rows = A.row_of_entries()
    off = rows != A.colidx
    S = sp.csr_matrix((A.vals[off], (rows[off], A.colidx[off])), shape=(A.n, A.n))
    rp = np.zeros(A.n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows[off], minlength=A.n), out=rp[1:])
    want = b - (S + sp.identity(A.n)) @ x
    got = oracle.residual(rp, A.colidx[off].astype(np.int32), A.vals[off], b, x, unit=True)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
