"""Differentiable sparse triangular solve.

``x = sparse_triangular_solve(plan, vals, b)`` solves A x = b with A the
plan's pattern carrying ``vals``.  The backward pass runs the adjoint solve
y = A^{-T} (dloss/dx) (the transposed CSR of Sec. 3.2, built once per plan)
and a sparse outer-product kernel on the stored pattern only: from eq. (1),
dx = -A^{-1} (dA) x, hence dloss/db = y and dloss/dA_ij = -y_i x_j.
"""
from __future__ import annotations

import torch

from .solver import TriangularPlan

# Algorithms that solve from the plan's level-ordered copy of the values.
COPYING_ALGOS = ("permuted", "blocked", "partitioned")


class _TriangularSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, plan, algo, transpose):
        if vals.data_ptr() != plan.vals.data_ptr():
            plan.set_values(vals)
        elif (plan.best_algo if algo == "auto" else algo) in COPYING_ALGOS:
            # the level-ordered copy is a snapshot: an in-place update of
            # `vals` (an optimizer step) keeps the pointer, so refresh it
            plan.refresh_values()
        x = plan.solve_transpose(b, algo=algo) if transpose else plan.solve(b, algo=algo)
        ctx.plan = plan
        ctx.algo = algo
        ctx.transpose = transpose
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        plan = ctx.plan
        gx = gx.contiguous()
        if ctx.transpose:
            # A^T x = b:  y = A^{-1} gx,  dloss/dA_ij = -x_i y_j
            y = plan.solve(gx, algo=ctx.algo)
            gv = plan.grad_vals(x, y) if ctx.needs_input_grad[0] else None
        else:
            y = plan.solve_transpose(gx, algo=ctx.algo)
            gv = plan.grad_vals(y, x) if ctx.needs_input_grad[0] else None
        gb = y if ctx.needs_input_grad[1] else None
        return gv, gb, None, None, None


def sparse_triangular_solve(plan: TriangularPlan, vals: torch.Tensor, b: torch.Tensor,
                            algo: str = "self", transpose: bool = False) -> torch.Tensor:
    """Differentiable x = A^{-1} b (or A^{-T} b) with A = (plan pattern, vals)."""
    return _TriangularSolve.apply(vals, b, plan, algo, transpose)


class SparseTriangularSolve(torch.nn.Module):
    """Module form: holds the pattern, analyses it on first use, and solves
    with whatever values tensor it is given."""

    def __init__(self, rowptr, colidx, upper=False, unit=False, algo="self"):
        super().__init__()
        self.register_buffer("rowptr", torch.as_tensor(rowptr, dtype=torch.int32))
        self.register_buffer("colidx", torch.as_tensor(colidx, dtype=torch.int32))
        self.upper, self.unit, self.algo = upper, unit, algo
        self._plan = None

    def plan_for(self, vals):
        if self._plan is None or self._plan.dtype != vals.dtype:
            self._plan = TriangularPlan(self.rowptr.contiguous(), self.colidx.contiguous(),
                                        vals.detach().contiguous(), self.upper, self.unit)
        return self._plan

    def forward(self, vals, b, transpose=False):
        return sparse_triangular_solve(self.plan_for(vals), vals, b, self.algo, transpose)
