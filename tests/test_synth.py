"""Checks on the input generators (shapes, structure, value recipe)."""
import numpy as np
import pytest

import synth


def generic_ilu0(A_dense):
    """Textbook IKJ ILU(0): Gaussian elimination that drops every update
    outside the pattern of A.  Returns (L unit lower, U upper) dense."""
    n = A_dense.shape[0]
    W = A_dense.copy()
    pat = A_dense != 0
    for i in range(1, n):
        for k in range(i):
            if not pat[i, k]:
                continue
            W[i, k] /= W[k, k]
            for j in range(k + 1, n):
                if pat[i, j]:
                    W[i, j] -= W[i, k] * W[k, j]
    return np.tril(W, -1) + np.eye(n), np.triu(W)


def laplacian_7pt_dense(nx, ny, nz):
    n = nx * ny * nz
    A = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                A[i, i] = 6.0
                for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    if x + dx < nx and y + dy < ny and z + dz < nz:
                        j = (x + dx) + nx * ((y + dy) + ny * (z + dz))
                        A[i, j] = A[j, i] = -1.0
    return A


def king_laplacian_dense(dims):
    """Graph Laplacian of the grid in which every point is joined to every
    point at Chebyshev distance 1 (the 9-point and 27-point stencils),
    built point by point."""
    n = int(np.prod(dims))
    A = np.zeros((n, n))
    coords = list(np.ndindex(*dims[::-1]))
    index = {c[::-1]: k for k, c in enumerate(coords)}
    for p, i in index.items():
        for q, j in index.items():
            if i != j and max(abs(a - b) for a, b in zip(p, q)) == 1:
                A[i, j] = -1.0
    np.fill_diagonal(A, 3 ** len(dims) - 1)
    return A


@pytest.mark.parametrize("dims,pts", [((4, 3), 9), ((3, 4, 2), 27), ((5, 4), 5),
                                      ((3, 3, 4), 7)])
def test_laplacian_triangles(dims, pts):
    L, U = synth.laplacian_triangles(dims, pts)
    check_csr(L)
    check_csr(U)
    Ld, Ud = L.scipy().toarray(), U.scipy().toarray()
    assert np.array_equal(np.triu(Ld, 1), 0 * Ld) and np.array_equal(np.tril(Ud, -1), 0 * Ud)
    np.testing.assert_array_equal(np.diag(Ld), np.diag(Ud))
    A = Ld + Ud - np.diag(np.diag(Ld))
    if pts in (9, 27):
        np.testing.assert_array_equal(A, king_laplacian_dense(dims))
    else:
        # 5/7 points: the axis neighbours only, diagonal 2 * dimensions
        assert np.all(np.diag(A) == 2 * len(dims))
        assert np.count_nonzero(A - np.diag(np.diag(A))) == 2 * (L.nnz - L.n)
    assert L.meta["points"] == pts and not L.upper and U.upper


def test_ilu0_factors_match_generic_ilu0():
    nx, ny, nz = 6, 5, 4
    Lw, Uw = generic_ilu0(laplacian_7pt_dense(nx, ny, nz))
    L, U = synth.lap3d_7pt_ilu0(nx, ny, nz)
    np.testing.assert_allclose(L.scipy().toarray(), Lw, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(U.scipy().toarray(), Uw, rtol=1e-14, atol=1e-14)
    assert L.unit and not U.unit and U.upper


def test_workload_shapes():
    A = synth.lap2d_5pt_lower(64, 64)
    assert A.n == 4096 and A.nnz == 12160
    L, U = synth.lap3d_7pt_ilu0(16, 16, 16)
    n = 16 ** 3
    assert L.nnz == U.nnz == n + 3 * (n - 16 * 16)


def check_csr(A):
    rows = A.row_of_entries()
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz
    assert np.all(np.diff(A.rowptr) >= 1)
    same_row = rows[1:] == rows[:-1]
    assert np.all(A.colidx[1:][same_row] > A.colidx[:-1][same_row])   # sorted, unique
    if A.upper:
        assert np.all(A.colidx >= rows)
    else:
        assert np.all(A.colidx <= rows)


def test_general_lower_recipe():
    A = synth.general_lower(200_000, seed=5)
    check_csr(A)
    lens = np.diff(A.rowptr)
    assert lens.max() <= 2000
    assert 14.5 < lens.mean() < 17.5                   # Pareto(2, 8) mean 16, minus clipping
    rows = A.row_of_entries()
    diag = A.colidx == rows
    assert diag.sum() == A.n                            # every diagonal stored
    off = ~diag
    assert np.all(np.abs(A.vals[off]) <= 1.0)
    absum = np.bincount(rows[off], weights=np.abs(A.vals[off]), minlength=A.n)
    np.testing.assert_allclose(A.vals[diag], 1.0 + absum, rtol=1e-15)
    dist = rows[off] - A.colidx[off]
    frac_band = np.mean(dist <= 512)
    assert 0.65 < frac_band < 0.80      # ~70% banded (duplicates redrawn) + uniform hits in band


def test_general_lower_deterministic():
    a = synth.general_lower(5000, seed=9)
    b = synth.general_lower(5000, seed=9)
    assert np.array_equal(a.colidx, b.colidx) and np.array_equal(a.vals, b.vals)


def test_block_diagonal_and_reversal():
    mats = synth.batch_general(5, seed=3, nmin=100, nmax=400)
    B = synth.block_diagonal(mats)
    check_csr(B)
    off = B.meta["offsets"]
    for s, m in enumerate(mats):
        r0, r1 = off[s], off[s + 1]
        sub = B.scipy()[r0:r1, r0:r1].toarray()
        np.testing.assert_array_equal(sub, m.scipy().toarray())
    U = synth.to_upper_by_reversal(mats[0])
    check_csr(U)
    n = mats[0].n
    P = np.eye(n)[::-1]
    np.testing.assert_array_equal(U.scipy().toarray(), P @ mats[0].scipy().toarray() @ P)


@pytest.mark.parametrize("count,seed", [(512, 1)])
def test_batch_sizes_log_uniform(count, seed):
    s = synth.batch_sizes(count, seed)
    assert s.min() >= 1000 and s.max() <= 65536
    assert abs(np.median(np.log(s)) - 0.5 * (np.log(1000) + np.log(65536))) < 0.4
