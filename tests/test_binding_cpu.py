"""Argument checks of the Python binding, on the host.  The library reads and
writes the tensors it is given through raw device pointers, so a tensor of
the wrong type, on the wrong device or with a layout other than the one the
call assumes must be refused before any call reaches the library (it would
be read or written out of bounds on the GPU).  The plan here is a stand-in
whose device is the CPU: every case below must raise ValueError before the
binding touches its (absent) handle."""
import pytest
import torch

from paper_1710_04985_gb300.solver import TriangularPlan

N = 6


@pytest.fixture
def plan():
    p = TriangularPlan.__new__(TriangularPlan)
    p.n, p.nnz, p.dtype, p.device = N, 11, torch.float64, torch.device("cpu")
    p.upper = p.unit = False
    p._h = None          # any call into the library would fail on it
    p._keep = [None, None, None]
    return p


def vec(dtype=torch.float64, device="cpu", n=N):
    return torch.zeros(n, dtype=dtype, device=device)


def mat(k, ld=None, dtype=torch.float64):
    ld = ld or k
    return torch.zeros(N, ld, dtype=dtype)[:, :k]


def test_solve_refuses_foreign_tensors(plan):
    for bad in (vec(torch.float32), vec(device="meta"), vec(n=N + 1), mat(2)[:, ::2]):
        with pytest.raises(ValueError):
            plan.solve(bad)
    for bad_out in (vec(torch.float32), vec(device="meta"), vec(n=N - 1)):
        with pytest.raises(ValueError):
            plan.solve(vec(), out=bad_out)
    with pytest.raises(ValueError):          # same columns, other leading dimension
        plan.solve(mat(2, 4), out=mat(2, 3))
    with pytest.raises(ValueError):
        plan.solve_transpose(vec(torch.float32))


def test_residual_and_refined_solve_check_every_array(plan):
    b = mat(2, 4)
    with pytest.raises(ValueError):          # x laid out unlike b
        plan.residual(b, mat(2))
    with pytest.raises(ValueError):
        plan.residual(b, mat(2, 4), out=mat(2))
    with pytest.raises(ValueError):
        plan.residual(b, mat(2, 4, torch.float32))
    with pytest.raises(ValueError):
        plan.residual(mat(2, 4, torch.float32), mat(2, 4))
    with pytest.raises(ValueError):          # FP64 right-hand side and solution only
        plan.solve_refined(vec(torch.float32))
    with pytest.raises(ValueError):
        plan.solve_refined(b, out=mat(2))
    with pytest.raises(ValueError):
        plan.solve_refined(vec(), out=vec(device="meta"))


def test_grad_vals_and_set_values_check_type_device_and_length(plan):
    with pytest.raises(ValueError):
        plan.grad_vals(vec(), vec(torch.float32))
    with pytest.raises(ValueError):
        plan.grad_vals(mat(2), mat(2, 3))
    with pytest.raises(ValueError):
        plan.grad_vals(vec(), vec(), out=torch.zeros(plan.nnz - 1, dtype=torch.float64))
    with pytest.raises(ValueError):
        plan.grad_vals(vec(), vec(), out=torch.zeros(plan.nnz, dtype=torch.float32))
    for bad in (torch.zeros(plan.nnz, dtype=torch.float32),
                torch.zeros(plan.nnz, dtype=torch.float64, device="meta"),
                torch.zeros(plan.nnz + 1, dtype=torch.float64)):
        with pytest.raises(ValueError):
            plan.set_values(bad)


def test_plan_refuses_host_or_mixed_device_arrays():
    rp = torch.tensor([0, 1], dtype=torch.int32)
    ci = torch.tensor([0], dtype=torch.int32)
    v = torch.ones(1, dtype=torch.float64)
    with pytest.raises(ValueError):
        TriangularPlan(rp, ci, v)            # host tensors


def test_block_diagonal_concatenates_and_refuses_inconsistent_systems():
    from paper_1710_04985_gb300.batch import block_diagonal
    sys0 = ([0, 1, 3], [0, 0, 1], [2.0, 1.0, 3.0])           # 2 x 2 lower
    sys1 = ([0, 1], [0], [5.0])                               # 1 x 1
    rp, ci, va, off = block_diagonal([sys0, sys1], device="cpu")
    assert rp.tolist() == [0, 1, 3, 4] and rp.dtype == torch.int32
    assert ci.tolist() == [0, 0, 1, 2] and ci.dtype == torch.int32
    assert va.tolist() == [2.0, 1.0, 3.0, 5.0] and off == [0, 2, 3]
    for bad in (([0, 1, 2], [0, 0, 1], [2.0, 1.0, 3.0]),     # rowptr ends short of colidx
                ([0, 1, 3], [0, 0, 1], [2.0, 1.0]),          # fewer values than entries
                ([1, 2, 4], [0, 0, 1], [2.0, 1.0, 3.0])):    # rowptr not from 0
        with pytest.raises(ValueError):
            block_diagonal([sys1, bad], device="cpu")
