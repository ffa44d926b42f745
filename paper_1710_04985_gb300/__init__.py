"""GB300-native sparse triangular solver after Li, "On Parallel Solution of
Sparse Triangular Linear Systems in CUDA" (arXiv:1710.04985).

Level-set analysis, a level-scheduled solve (Alg. 1) and a self-scheduled
solve (Alg. 3) for CSR ``Lx = b`` / ``Ux = b`` on sm_103a, behind the C ABI of
``include/sptrsv.h``; plus the adjoint solve and sparse gradient
(``autograd``), batched graph-replayed solves with an autotuner (``batch``,
``autotune``) and FP32 solves with FP64 iterative refinement
(``TriangularPlan.solve_refined``).
"""
from .solver import TriangularPlan, plan_from_arrays, SptrsvError  # noqa: F401
from .autograd import sparse_triangular_solve, SparseTriangularSolve  # noqa: F401
from .batch import BatchedTriangularSolve, block_diagonal  # noqa: F401
from . import autotune  # noqa: F401
