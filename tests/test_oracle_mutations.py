"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped or wrong term, a wrong sign, index or
direction, a transposed operand, an off-by-one level, an unstable order) in a
copy of the oracle's C source, compiles it, swaps it in for the oracle, and
runs the pin tests: at least one of them must fail.  The real oracle passes
the same pins (tests/test_oracle_pins.py)."""
import ctypes
import os

import pytest

import oracle
from oracle import build as oracle_build
import test_oracle_pins as pins

SRC = open(oracle_build.SRC).read()

MUTATIONS = {
    "divide_by_diag_replaced_by_multiply": (
        "x[(size_t)i * ldx + c] = unit ? s : s / d;", "x[(size_t)i * ldx + c] = unit ? s : s * d;"),
    "subtraction_sign_flipped": (
        "s -= vals[p] * x[(size_t)j * ldx + c];", "s += vals[p] * x[(size_t)j * ldx + c];"),
    "dependency_index_replaced_by_row": (
        "s -= vals[p] * x[(size_t)j * ldx + c];", "s -= vals[p] * x[(size_t)i * ldx + c];"),
    "unit_flag_ignored_in_solve": (
        "const double *b, int ldb, double *x, int ldx)\n{\n    for (int c = 0; c < k; ++c) {",
        "const double *b, int ldb, double *x, int ldx)\n{\n    unit = 0;\n    for (int c = 0; c < k; ++c) {"),
    "upper_sweep_in_forward_order": (
        "            int i = upper ? n - 1 - t : t;\n            double s = b",
        "            int i = t;\n            double s = b"),
    "level_off_by_one": ("lev[i] = best + 1;", "lev[i] = best + 2;"),
    "level_min_instead_of_max": ("if (lev[j] > best) best = lev[j];",
                                 "if (lev[j] < best) best = lev[j];"),
    "transposed_levels_without_max": ("if (lev[j] + 1 > lev[i]) lev[i] = lev[j] + 1;",
                                      "lev[i] = lev[j] + 1;"),
    "level_sets_unstable_order": (
        "    for (int i = 0; i < n; ++i) {\n        int m = lev[i];",
        "    for (int i = n - 1; i >= 0; --i) {\n        int m = lev[i];"),
    "transpose_sweep_sign_flipped": ("y[(size_t)i * ldy + c] -= vals[p] * yj;",
                                     "y[(size_t)i * ldy + c] += vals[p] * yj;"),
    "transpose_sweep_skips_diagonal_division": ("double yj = y[(size_t)j * ldy + c] / d;",
                                                "double yj = y[(size_t)j * ldy + c];"),
    "gradient_sign_flipped": ("gvals[p] = -s;", "gvals[p] = s;"),
    "gradient_operands_transposed": (
        "s += y[(size_t)i * ldy + c] * x[(size_t)j * ldx + c];",
        "s += y[(size_t)j * ldy + c] * x[(size_t)i * ldx + c];"),
    "residual_drops_unit_diagonal": ("if (unit) s -= x[(size_t)i * ldx + c];", ""),
    "residual_sign_flipped": ("s -= x[(size_t)j * ldx + c] * vals[p];",
                              "s += x[(size_t)j * ldx + c] * vals[p];"),
    "residual_uses_stored_unit_diagonal": ("if (unit && j == i) continue;", ""),
}

PIN_CHECKS = [
    lambda: [pins.test_solve_matches_dense_lapack(n, up, un)
             for n in (2, 7, 33, 64) for up in (False, True) for un in (False, True)],
    lambda: [pins.test_solve_transpose_matches_dense_lapack(n, up, un)
             for n in (5, 40) for up in (False, True) for un in (False, True)],
    pins.test_manufactured_solution_workload0,
    lambda: pins.test_levels_closed_form_2d(13, 4),
    lambda: pins.test_levels_closed_form_3d((6, 5, 4)),
    pins.test_fig1_worked_example,
    lambda: [pins.test_levels_brute_force(sd, up) for sd in range(3) for up in (False, True)],
    pins.test_levels_transpose_equal_levels_of_explicit_transpose,
    pins.test_level_sets_are_a_stable_counting_sort,
    pins.test_adjoint_identity,
    lambda: [pins.test_gradient_finite_differences(up, un)
             for up in (False, True) for un in (False, True)],
    pins.test_gradient_matches_dense_outer_product,
    pins.test_residual_matches_scipy,
]


def run_pins():
    failed = 0
    for check in PIN_CHECKS:
        try:
            check()
        except AssertionError:
            failed += 1
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, "mutation anchor must be unique"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    oracle_build.build(src=str(src), out=so)
    real = oracle._load()
    try:
        oracle._lib = oracle._bind(ctypes.CDLL(so))
        assert run_pins() > 0, f"no pin caught '{name}'"
    finally:
        oracle._lib = real


def test_real_oracle_passes_the_same_checks():
    oracle._load()
    assert run_pins() == 0
