"""Seeded synthetic inputs shaped like the workloads of Li, arXiv:1710.04985.

This module only BUILDS inputs: sparsity patterns, matrix values and vectors.
It holds none of the solver's arithmetic (no levels, no substitution).  The
CPU oracle and the CUDA path both take their inputs from here, which is the
only code they share.

Matrices are CSR with the diagonal stored in its row, sorted column indices,
0-based int32 indices and float64 values.

Workloads (seeds are ``SEED_BASE + k`` for workload k):

* ``lap2d_5pt_lower``    lower triangle of the 2-D 5-point Laplacian (Sec. 5.1,
                         Table 2), diagonal 4, off-diagonals -1.
* ``lap3d_7pt_ilu0``     ILU(0) factors of the 3-D 7-point Laplacian in natural
                         order (Sec. 5.1, Table 2; ILU named in Sec. 1).
* ``general_lower``      general sparse lower triangle standing in for the
                         SuiteSparse/MFEM matrices of Sec. 5.2 (Table 3), which
                         are not available: Pareto row lengths, banded plus
                         uniform column draws, diagonally dominant values.
* ``laplacian_triangles`` lower and upper triangles (diagonal included) of the
                         5/9-point 2-D and 7/27-point 3-D Laplacians on the
                         regular grids of Table 2 (Sec. 5.1).
* ``block_diagonal``     many independent systems concatenated into one.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

SEED_BASE = 1710049850


@dataclass
class CSR:
    """A square triangular matrix in CSR, diagonal stored in its row."""

    n: int
    rowptr: np.ndarray          # int32 [n + 1]
    colidx: np.ndarray          # int32 [nnz]
    vals: np.ndarray            # float64 [nnz]
    upper: bool = False
    unit: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def with_vals(self, vals) -> "CSR":
        return replace(self, vals=np.ascontiguousarray(vals))

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colidx, self.rowptr),
                             shape=(self.n, self.n))

    def row_of_entries(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.rowptr))


def _from_sorted_coo(n, rows, cols, vals, **kw) -> CSR:
    """CSR from COO entries already sorted by (row, col)."""
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31, "nnz must fit int32"
    return CSR(n, rowptr.astype(np.int32), np.ascontiguousarray(cols, dtype=np.int32),
               np.ascontiguousarray(vals, dtype=np.float64), **kw)


def _stencil_triangle(dims, offsets, upper):
    """Sorted COO (rows, cols, which-offset) of the entries of a structured
    grid operator whose neighbour offsets are ``offsets`` (lists of per-axis
    displacements, axis 0 fastest), restricted to one triangle including the
    diagonal.  Lexicographic ordering, x fastest."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]   # axis 0 = x
    strides = np.cumprod((1,) + dims[:-1])
    deltas = [int(sum(o * s for o, s in zip(off, strides))) for off in offsets]
    keep = [k for k, d in enumerate(deltas) if (d <= 0 if not upper else d >= 0)]
    keep.sort(key=lambda k: deltas[k])          # ascending column within a row
    lin = np.arange(n, dtype=np.int64)
    cols = np.empty((n, len(keep)), dtype=np.int64)
    ok = np.ones((n, len(keep)), dtype=bool)
    for slot, k in enumerate(keep):
        cols[:, slot] = lin + deltas[k]
        for ax, o in enumerate(offsets[k]):
            if o:
                c = coords[ax] + o
                ok[:, slot] &= (c >= 0) & (c < dims[ax])
    kinds = np.broadcast_to(np.array(keep, dtype=np.int16), cols.shape)
    rows = np.broadcast_to(lin[:, None], cols.shape)
    return n, rows[ok], cols[ok], kinds[ok]


_FIVE_POINT = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
_SEVEN_POINT = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def lap2d_5pt_lower(nx: int, ny: int) -> CSR:
    """Lower triangle, diagonal included, of the 5-point Laplacian on an
    ``nx`` x ``ny`` grid in lexicographic order: diagonal 4, neighbours -1."""
    n, rows, cols, _ = _stencil_triangle((nx, ny), _FIVE_POINT, upper=False)
    vals = np.where(rows == cols, 4.0, -1.0)
    return _from_sorted_coo(n, rows, cols, vals, upper=False,
                            name=f"lap2d_5pt_lower_{nx}x{ny}",
                            meta={"grid": (nx, ny)})


def lap2d_5pt_upper(nx: int, ny: int) -> CSR:
    """Upper triangle, diagonal included, of the same 5-point operator."""
    n, rows, cols, _ = _stencil_triangle((nx, ny), _FIVE_POINT, upper=True)
    vals = np.where(rows == cols, 4.0, -1.0)
    return _from_sorted_coo(n, rows, cols, vals, upper=True,
                            name=f"lap2d_5pt_upper_{nx}x{ny}",
                            meta={"grid": (nx, ny)})


def lap3d_7pt_ilu0_pivots(nx: int, ny: int, nz: int) -> np.ndarray:
    """Pivots u_ii of ILU(0) of the 7-point Laplacian (diagonal 6,
    neighbours -1) in natural order.

    With no fill allowed, the IKJ elimination only ever updates the diagonal:
    u_ii = 6 - sum over the lower neighbours k of i of 1/u_kk.  Points on one
    anti-diagonal plane x+y+z = const depend only on the previous plane, so
    the recurrence is evaluated plane by plane."""
    u = np.zeros((nz, ny, nx), dtype=np.float64)
    z, y, x = np.indices((nz, ny, nx))
    d = (x + y + z).reshape(-1)
    order = np.argsort(d, kind="stable")
    bounds = np.searchsorted(d[order], np.arange(nx + ny + nz - 1))
    bounds = np.append(bounds, d.size)
    zf, yf, xf = z.reshape(-1), y.reshape(-1), x.reshape(-1)
    flat = u.reshape(-1)
    for w in range(nx + ny + nz - 2):
        idx = order[bounds[w]:bounds[w + 1]]
        acc = np.full(idx.shape, 6.0)
        for ok, nb in ((xf[idx] > 0, idx - 1),
                       (yf[idx] > 0, idx - nx),
                       (zf[idx] > 0, idx - nx * ny)):
            acc[ok] -= 1.0 / flat[nb[ok]]
        flat[idx] = acc
    return flat


def lap3d_7pt_ilu0(nx: int, ny: int, nz: int):
    """ILU(0) factors ``(L, U)`` of the 7-point Laplacian on an
    ``nx`` x ``ny`` x ``nz`` grid, natural ordering.

    L is unit lower triangular and STORES its unit diagonal explicitly
    (L_ik = -1/u_kk for the lower neighbours k); U is upper triangular with
    U_ii = u_ii and U_ij = -1 for the upper neighbours j.  Both have the
    pattern of the matching triangle of the Laplacian."""
    piv = lap3d_7pt_ilu0_pivots(nx, ny, nz)
    n, rows, cols, _ = _stencil_triangle((nx, ny, nz), _SEVEN_POINT, upper=False)
    lvals = np.where(rows == cols, 1.0, -1.0 / piv[cols])
    L = _from_sorted_coo(n, rows, cols, lvals, upper=False, unit=True,
                         name=f"ilu0_L_7pt_{nx}x{ny}x{nz}",
                         meta={"grid": (nx, ny, nz)})
    n, rows, cols, _ = _stencil_triangle((nx, ny, nz), _SEVEN_POINT, upper=True)
    uvals = np.where(rows == cols, piv[rows], -1.0)
    U = _from_sorted_coo(n, rows, cols, uvals, upper=True, unit=False,
                         name=f"ilu0_U_7pt_{nx}x{ny}x{nz}",
                         meta={"grid": (nx, ny, nz)})
    return L, U


def lap3d_7pt_lower(nx: int, ny: int, nz: int) -> CSR:
    """Lower triangle of the 7-point Laplacian itself (diagonal 6)."""
    n, rows, cols, _ = _stencil_triangle((nx, ny, nz), _SEVEN_POINT, upper=False)
    vals = np.where(rows == cols, 6.0, -1.0)
    return _from_sorted_coo(n, rows, cols, vals, name=f"lap3d_7pt_lower_{nx}x{ny}x{nz}",
                            meta={"grid": (nx, ny, nz)})


def _full_stencil(ndim: int):
    """Every displacement in {-1, 0, 1}^ndim: the 9-point (2-D) and 27-point
    (3-D) stencils of Sec. 5.1, diagonal included."""
    grids = np.indices((3,) * ndim).reshape(ndim, -1).T - 1
    return [tuple(int(v) for v in g) for g in grids]


STENCILS = {
    (2, 5): _FIVE_POINT,
    (2, 9): _full_stencil(2),
    (3, 7): _SEVEN_POINT,
    (3, 27): _full_stencil(3),
}


def laplacian_triangles(dims, points: int):
    """``(L + D, U + D)`` of the ``points``-point Laplacian on a regular grid
    ``dims = (nx, ny)`` or ``(nx, ny, nz)`` in lexicographic order (x
    fastest), the test problems of Sec. 5.1 (Table 2) split as in eq. (3):
    A = L + D + U.  Every neighbour entry is -1 and the diagonal is
    ``points - 1`` (the number of neighbours of an interior point), so A is
    the graph Laplacian of the stencil: 4/-1 for 5 points, 8/-1 for 9,
    6/-1 for 7 and 26/-1 for 27."""
    dims = tuple(int(d) for d in dims)
    offsets = STENCILS[(len(dims), int(points))]
    diag = float(points - 1)
    tag = "x".join(str(d) for d in dims)
    out = []
    for upper in (False, True):
        n, rows, cols, _ = _stencil_triangle(dims, offsets, upper=upper)
        vals = np.where(rows == cols, diag, -1.0)
        out.append(_from_sorted_coo(n, rows, cols, vals, upper=upper,
                                    name=f"lap{len(dims)}d_{points}pt_"
                                         f"{'upper' if upper else 'lower'}_{tag}",
                                    meta={"grid": dims, "points": int(points)}))
    return out[0], out[1]


# Regular grids of Table 2 (Sec. 5.1): n = 2^20 in 2-D and 2^21 in 3-D, with
# growing aspect ratios rho_yx = ny/nx and rho_zx = nz/nx (eq. (5)).
TABLE2_GRIDS_2D = [(1024, 1024), (512, 2048), (256, 4096), (128, 8192), (64, 16384)]
TABLE2_GRIDS_3D = [(128, 128, 128), (64, 128, 256), (64, 64, 512), (32, 64, 1024),
                   (32, 32, 2048)]


def general_lower(n: int, seed: int, band: int = 512, p_band: float = 0.7,
                  xm: float = 8.0, maxlen: int = 2000) -> CSR:
    """General sparse lower triangle, diagonally dominant.

    Row i holds ``len_i = min(maxlen, i + 1, rint(xm / sqrt(U)))`` entries
    (U uniform on (0, 1]; a Pareto law with shape 2 and scale xm, mean 2 xm)
    including its diagonal.  Each of the ``len_i - 1`` off-diagonal columns is
    drawn, with probability ``p_band``, uniformly from the band
    ``[max(0, i - band), i - 1]`` (uniformly from all earlier columns once the
    band is used up), otherwise uniformly from ``[0, i - 1]``; duplicates are
    redrawn.  Rows that want at least half of the earlier columns sample them
    uniformly without replacement.  Off-diagonal values are uniform on
    [-1, 1] and the diagonal is ``1 + sum |off-diagonals|``."""
    rng = np.random.default_rng(seed)
    i_all = np.arange(n, dtype=np.int64)
    u = 1.0 - rng.random(n)
    length = np.minimum(np.minimum(maxlen, i_all + 1), np.rint(xm / np.sqrt(u)))
    m = length.astype(np.int64) - 1                      # 0 <= m <= i

    dense_rows = np.nonzero((m > 0) & (2 * m >= i_all))[0]
    sparse_rows = np.nonzero((m > 0) & (2 * m < i_all))[0]

    key_parts = []
    for r in dense_rows:
        c = rng.choice(int(r), size=int(m[r]), replace=False)
        key_parts.append(int(r) * n + np.sort(c).astype(np.int64))

    need = np.zeros(n, dtype=np.int64)
    need[sparse_rows] = m[sparse_rows]
    bandsize = np.minimum(band, i_all)
    inband = np.zeros(n, dtype=np.int64)
    accepted = []                 # sorted int64 key arrays, disjoint
    active = sparse_rows
    while active.size:
        r = np.repeat(active, need[active])
        full = inband[r] >= bandsize[r]
        use_band = (rng.random(r.size) < p_band) & ~full
        uu = rng.random(r.size)
        lo = np.maximum(0, r - band)
        c = np.where(use_band, lo + np.floor(uu * (r - lo)),
                     np.floor(uu * r)).astype(np.int64)
        c = np.minimum(c, r - 1)
        cand = np.sort(r * n + c)
        if cand.size:
            cand = cand[np.concatenate(([True], cand[1:] != cand[:-1]))]
        for prev in accepted:
            if prev.size == 0:
                continue
            pos = np.searchsorted(prev, cand)
            pos = np.minimum(pos, prev.size - 1)
            cand = cand[prev[pos] != cand]
        accepted.append(cand)
        cr = cand // n
        cc = cand - cr * n
        got = np.bincount(cr, minlength=n)
        need -= got
        inband += np.bincount(cr, weights=(cc >= cr - band), minlength=n).astype(np.int64)
        active = np.nonzero(need > 0)[0]
        if len(accepted) > 4:     # keep the membership checks cheap
            accepted = [np.sort(np.concatenate(accepted))]

    diag_keys = i_all * n + i_all
    keys = np.sort(np.concatenate(key_parts + accepted + [diag_keys]))
    rows = keys // n
    cols = keys - rows * n
    offd = rows != cols
    vals = np.empty(keys.size, dtype=np.float64)
    vals[offd] = rng.uniform(-1.0, 1.0, int(offd.sum()))
    absum = np.bincount(rows[offd], weights=np.abs(vals[offd]), minlength=n)
    vals[~offd] = 1.0 + absum[rows[~offd]]
    return _from_sorted_coo(n, rows, cols, vals, upper=False,
                            name=f"general_lower_n{n}_s{seed}",
                            meta={"seed": seed, "band": band, "p_band": p_band})


def to_upper_by_reversal(A: CSR) -> CSR:
    """The upper triangle P A P (P the reversal permutation) of a lower CSR:
    row i of the result is row n-1-i of A with columns mirrored."""
    n = A.n
    rows = A.row_of_entries().astype(np.int64)
    nr = n - 1 - rows
    nc = n - 1 - A.colidx.astype(np.int64)
    order = np.lexsort((nc, nr))
    return _from_sorted_coo(n, nr[order], nc[order], A.vals[order], upper=True,
                            unit=A.unit, name=A.name + "_reversed", meta=dict(A.meta))


def block_diagonal(mats) -> CSR:
    """Concatenate independent systems (all lower or all upper) into one
    block-diagonal CSR; ``meta['offsets']`` gives each system's first row."""
    mats = list(mats)
    assert mats and all(m.upper == mats[0].upper for m in mats)
    offsets = np.zeros(len(mats) + 1, dtype=np.int64)
    np.cumsum([m.n for m in mats], out=offsets[1:])
    nnz_off = np.zeros(len(mats) + 1, dtype=np.int64)
    np.cumsum([m.nnz for m in mats], out=nnz_off[1:])
    assert offsets[-1] < 2**31 and nnz_off[-1] < 2**31
    rowptr = np.concatenate([m.rowptr[:-1].astype(np.int64) + nnz_off[s]
                             for s, m in enumerate(mats)] + [nnz_off[-1:]])
    colidx = np.concatenate([m.colidx.astype(np.int64) + offsets[s]
                             for s, m in enumerate(mats)])
    vals = np.concatenate([m.vals for m in mats])
    return CSR(int(offsets[-1]), rowptr.astype(np.int32), colidx.astype(np.int32),
               vals, upper=mats[0].upper, unit=mats[0].unit,
               name=f"block_diagonal_{len(mats)}",
               meta={"offsets": offsets, "nnz_offsets": nnz_off})


def batch_sizes(count: int, seed: int, nmin: int = 1000, nmax: int = 65536) -> np.ndarray:
    """System sizes log-uniform on [nmin, nmax]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))).astype(np.int64)


def batch_general(count: int, seed: int, nmin: int = 1000, nmax: int = 65536):
    """``count`` independent ``general_lower`` systems; system s uses seed
    ``seed + 1 + s`` and a size from ``batch_sizes(count, seed, ...)``."""
    sizes = batch_sizes(count, seed, nmin, nmax)
    return [general_lower(int(nk), seed + 1 + s) for s, nk in enumerate(sizes)]


def _general_lower_args(args):
    return general_lower(*args)


def batch_general_parallel(count: int, seed: int, nmin: int = 1000, nmax: int = 65536,
                           processes: int = 0):
    """``batch_general`` generated in worker processes (spawned, so safe to
    call after CUDA is initialised); same matrices, same order."""
    import multiprocessing as mp
    import os
    sizes = batch_sizes(count, seed, nmin, nmax)
    jobs = [(int(nk), seed + 1 + s) for s, nk in enumerate(sizes)]
    procs = processes or min(16, os.cpu_count() or 1)
    if procs <= 1:
        return [general_lower(*j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_general_lower_args, jobs, chunksize=4)


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def times_vector(A: CSR, x: np.ndarray) -> np.ndarray:
    """A @ x through scipy (manufactured right-hand sides b = A x_true);
    a unit-diagonal matrix is applied with its diagonal taken as 1."""
    M = A.scipy()
    if A.unit:
        import scipy.sparse as sp
        d = M.diagonal()
        M = M - sp.diags(d) + sp.identity(A.n, format="csr")
    return M @ x


# ---------------------------------------------------------------- workloads

def workload0():
    """64 x 64 5-point lower triangle; x_true ~ U[-1,1]; b = L x_true."""
    A = lap2d_5pt_lower(64, 64)
    xt = uniform(A.n, SEED_BASE + 0)
    return A, xt, times_vector(A, xt)


def workload1(nx: int = 128, ny: int = 128, nz: int = 128):
    """ILU(0) factors of the 128^3 7-point Laplacian, with x_true ~ U[-1,1]
    and manufactured right-hand sides for each factor."""
    L, U = lap3d_7pt_ilu0(nx, ny, nz)
    xt = uniform(L.n, SEED_BASE + 1)
    return L, U, xt, times_vector(L, xt), times_vector(U, xt)


def workload2(n: int = 1_000_000):
    """General lower triangle, n = 10^6; x_true ~ U[-1,1], b = A x_true."""
    A = general_lower(n, SEED_BASE + 2)
    xt = uniform(n, SEED_BASE + 2 + 7919)
    return A, xt, times_vector(A, xt)
