"""Batches of independent systems on the partitioned solve (CUDA path vs the
CPU oracle, through the C ABI).

A block-diagonal batch decouples at every system boundary: no row of a later
system depends on a row of an earlier one.  The partitioned solve finds
these boundaries itself, cuts long systems into balanced parts, packs short
neighbouring systems into one part and hands the parts out latest start
first (a system's slack behind the deepest one plus the piece's share of the
system's levels).  The tests check that layout against the systems the batch
was built from, and every solution against the oracle's solve of each system
alone.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL32, TOL64, dev, plan_for, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_device):
    yield


def _batch(count, seed, nmin, nmax, upper=False):
    mats = synth.batch_general(count, seed=seed, nmin=nmin, nmax=nmax)
    if upper:
        mats = [synth.to_upper_by_reversal(m) for m in mats]
    return mats, synth.block_diagonal(mats)


def _system_of_rows(offsets, n):
    sys_of = np.zeros(n, dtype=np.int64)
    for s in range(len(offsets) - 1):
        sys_of[offsets[s]:offsets[s + 1]] = s
    return sys_of


def _check_layout(info, mats, offsets, S, upper):
    """Parts never split a system except into pieces of a system longer than
    S/2; short systems are only packed whole; the hand-out order is by the
    latest start level of a part, (deepest level - depth of its system) +
    piece index * levels of its system // parts of its system, then order of
    substitution, so a system's pieces follow its order of substitution."""
    n = int(offsets[-1])
    sizes = np.diff(offsets)
    sys_of = _system_of_rows(offsets, n)
    depth = np.array([oracle.levels(m.rowptr, m.colidx, upper=m.upper)[1] for m in mats])
    pp = info["part_ptr"].cpu().numpy()
    order = info["order"].cpu().numpy()
    assert info["nblocks"] == len(mats)
    assert info["nparts"] == len(pp) - 1 and pp[0] == 0 and pp[-1] == n
    assert np.all(np.diff(pp) >= 1)
    assert info["max_part_rows"] == np.diff(pp).max() <= S
    assert np.array_equal(np.sort(order), np.arange(n))
    parts = []
    for j in range(info["nparts"]):
        rows = order[pp[j]:pp[j + 1]]
        ss = np.unique(sys_of[rows])
        if len(ss) > 1:          # packed: only whole short systems
            assert np.all(sizes[ss] <= S // 2)
            assert len(rows) == sizes[ss].sum()
        else:
            s = ss[0]
            if len(rows) < sizes[s]:
                assert sizes[s] > S // 2
        # position in substitution order of the part's first row
        first = rows.max() if upper else rows.min()
        sub = n - 1 - first if upper else first
        parts.append((sys_of[first], sub))
    # piece index: rank of the part among its system's parts in substitution order
    piece = [sum(1 for s2, u in parts if s2 == s and u < sub) for s, sub in parts]
    count = [sum(1 for s2, _ in parts if s2 == s) for s, _ in parts]
    maxlev = int(depth.max()) - 1
    keys = [((maxlev - (int(depth[s]) - 1)) + piece[j] * int(depth[s]) // count[j], sub)
            for j, (s, sub) in enumerate(parts)]
    assert keys == sorted(keys)
    for s in set(s for s, _ in parts):   # a system's pieces in substitution order
        subs = [sub for s2, sub in parts if s2 == s]
        assert subs == sorted(subs)


@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("S", [1500, 4096, 0])
def test_partitioned_batch_layout_and_parity(upper, S):
    mats, A = _batch(36, 41, 200, 6000, upper=upper)
    offsets = A.meta["offsets"]
    b = synth.uniform(A.n, 43)
    with plan_for(A) as p:
        bt = torch.tensor(b, device=dev())
        p.set_tuning(1, 256, 0)
        ref_self = p.solve(bt, algo="self")
        p.set_partition(S, 1)
        x = p.solve(bt, algo="partitioned")
        assert torch.equal(x, ref_self)       # same fold order as the in-place form
        xs = x.cpu().numpy()
        for s, m in enumerate(mats):
            ref = oracle.solve(m.rowptr, m.colidx, m.vals, b[offsets[s]:offsets[s + 1]],
                               upper=m.upper)
            assert relerr(xs[offsets[s]:offsets[s + 1]], ref) <= TOL64
        info = p.partition_info()
        _check_layout(info, mats, offsets, p.partition, upper)
        for cl in (2, 4):                     # clusters over parts of uneven length
            p.set_partition(S, cl)
            assert torch.equal(p.solve(bt, algo="partitioned"), ref_self), cl
        assert p.status() == (0, -1)


def test_partitioned_batch_transpose_and_fp32():
    mats, A = _batch(20, 47, 500, 5000)
    offsets = A.meta["offsets"]
    g = synth.uniform(A.n, 49)
    with plan_for(A) as p:
        p.set_partition(2048, 1)
        y = p.solve_transpose(torch.tensor(g, device=dev()), algo="partitioned").cpu().numpy()
        info = p.partition_info(transpose=True)
        assert info["nblocks"] == len(mats)
        for s, m in enumerate(mats):
            ref = oracle.solve_transpose(m.rowptr, m.colidx, m.vals, g[offsets[s]:offsets[s + 1]])
            assert relerr(y[offsets[s]:offsets[s + 1]], ref) <= TOL64
    with plan_for(A, dtype=torch.float32) as p:
        p.set_partition(3000, 2)
        b = synth.uniform(A.n, 53)
        x = p.solve(torch.tensor(b, device=dev(), dtype=torch.float32),
                    algo="partitioned").cpu().numpy()
        for s, m in enumerate(mats):
            ref = oracle.solve(m.rowptr, m.colidx, m.vals, b[offsets[s]:offsets[s + 1]])
            assert relerr(x[offsets[s]:offsets[s + 1]].astype(np.float64), ref) <= TOL32


def test_partitioned_many_one_row_blocks():
    """A diagonal matrix decouples at every row: parts pack rows by windows of
    S/2 positions."""
    n = 5003
    rows = np.arange(n)
    A = synth._from_sorted_coo(n, rows, rows, 1.0 + np.arange(n) % 7, upper=False)
    b = synth.uniform(n, 57)
    with plan_for(A) as p:
        p.set_partition(64, 1)
        x = p.solve(torch.tensor(b, device=dev()), algo="partitioned")
        assert relerr(x, b / A.vals) <= TOL64
        info = p.partition_info()
        assert info["nblocks"] == n
        assert info["max_part_rows"] <= 64
        assert info["nparts"] == -(-n // 32)
