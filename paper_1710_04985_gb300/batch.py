"""Many independent triangular systems in one self-scheduled launch.

The systems (uneven sizes, all lower or all upper) are concatenated into one
block-diagonal CSR, analysed once, tuned by the autotuner, and solved by one
persistent self-scheduled launch that a CUDA graph replays.  Rows of
different systems never wait on one another, so the level sets of the batch
are the union of the per-system level sets and the launch overlaps the
systems' dependency chains.  The partitioned form finds the system
boundaries itself (the matrix decouples there): its parts never mix a piece
of one system with another, and the deepest systems are started first.

``solve_refined`` solves the same batch with FP32 bulk solves and FP64
iterative refinement (the precision form), one refinement loop for all
systems together.
"""
from __future__ import annotations

import torch

from . import _lib, autotune
from .solver import TriangularPlan


def block_diagonal(systems, device="cuda", dtype=torch.float64):
    """Concatenate CSR systems ``[(rowptr, colidx, vals), ...]`` into one
    block-diagonal CSR on `device`.  Returns (rowptr, colidx, vals, offsets)
    with ``offsets[s]`` the first row of system s."""
    rps, cis, vas, sizes, nnzs = [], [], [], [], []
    for s, (rp, ci, va) in enumerate(systems):
        rp = torch.as_tensor(rp).to(device=device, dtype=torch.int64)
        rps.append(rp)
        cis.append(torch.as_tensor(ci).to(device=device, dtype=torch.int64))
        vas.append(torch.as_tensor(va).to(device=device, dtype=dtype))
        if rp.dim() != 1 or rp.numel() < 1:
            raise ValueError(f"system {s}: rowptr must be a vector of n + 1 entries")
        sizes.append(rp.numel() - 1)
        nnzs.append(int(rp[-1].item()))
        # the offsets below shift every system by the entries of the ones before
        if int(rp[0].item()) != 0 or nnzs[-1] != cis[-1].numel() or \
                cis[-1].numel() != vas[-1].numel():
            raise ValueError(f"system {s}: rowptr must run from 0 to the number of entries, "
                             "and colidx and vals must hold that many")
    offsets = [0]
    nnz_off = [0]
    for nk, zk in zip(sizes, nnzs):
        offsets.append(offsets[-1] + nk)
        nnz_off.append(nnz_off[-1] + zk)
    if offsets[-1] > _lib.MAX_SIZE or nnz_off[-1] > _lib.MAX_SIZE:
        raise ValueError("batch larger than the solver's index range (SPTRSV_MAX_SIZE)")
    rowptr = torch.cat([rp[:-1] + nnz_off[s] for s, rp in enumerate(rps)] +
                       [torch.tensor([nnz_off[-1]], device=device, dtype=torch.int64)])
    colidx = torch.cat([ci + offsets[s] for s, ci in enumerate(cis)])
    vals = torch.cat(vas)
    return (rowptr.to(torch.int32).contiguous(), colidx.to(torch.int32).contiguous(),
            vals.contiguous(), offsets)


class BatchedTriangularSolve:
    """One plan over a block-diagonal batch, solved by one graph replay."""

    def __init__(self, systems, upper=False, unit=False, nrhs=1, dtype=torch.float64,
                 device="cuda", tune=True):
        rowptr, colidx, vals, offsets = block_diagonal(systems, device, dtype)
        self.offsets = offsets
        self.nrhs = nrhs
        self.plan = TriangularPlan(rowptr, colidx, vals, upper=upper, unit=unit)
        n = self.plan.n
        shape = (n,) if nrhs == 1 else (n, nrhs)
        self.b = torch.zeros(shape, dtype=dtype, device=device)
        self.x = torch.empty_like(self.b)
        self.tuning = None
        if tune:
            self.b.uniform_(-1, 1)
            self.tuning = autotune.tune_algos(self.plan, self.b, self.x)
        self.graph = None

    @property
    def n(self):
        return self.plan.n

    def capture(self):
        """Record the solve of self.b into self.x as a CUDA graph."""
        self.plan.solve(self.b, out=self.x, algo="auto")   # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.plan.solve(self.b, out=self.x, algo="auto")
        self.graph = g
        return g

    def solve(self, b=None):
        """Solve every system; `b` (optional) is copied into the static input."""
        if b is not None:
            self.b.copy_(b)
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.x

    def solve_refined(self, b=None, max_iter=10, tol=8 * 2.0 ** -52):
        """Every system by FP32 solves (the tuned form) with FP64 residuals
        and updates; returns ``(x, corrections, relative_residual)``.  FP64
        batches only; not captured in a graph (each refinement step reads
        the residual norm on the host)."""
        if b is not None:
            self.b.copy_(b)
        return self.plan.solve_refined(self.b, out=self.x, max_iter=max_iter, tol=tol)

    def split(self, x=None):
        x = self.x if x is None else x
        return [x[self.offsets[s]:self.offsets[s + 1]] for s in range(len(self.offsets) - 1)]
