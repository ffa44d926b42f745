"""CPU-only checks of the C ABI: the library loads, exports every entry point
that include/sptrsv.h declares, the binding covers them, and the host-side
argument checks answer without touching a GPU.  Also checks that the oracle
and the CUDA path share no code."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sptrsv.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPTRSV_API\s+[\w\s\*]*?\b(sptrsv_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_04985_gb300 import _lib, build
    path = build.library_path()
    if not os.path.exists(path):
        build.build()
    return _lib.load()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("sptrsv_analyze", "sptrsv_solve", "sptrsv_solve_transpose", "sptrsv_free"):
        assert core in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    from paper_1710_04985_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    # nothing but the C ABI is exported
    assert all(s.startswith("sptrsv_") for s in exported), sorted(exported)


def test_binding_covers_the_header(lib):
    from paper_1710_04985_gb300 import _lib
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert bound == set(declared_functions())
    for name in bound:
        assert hasattr(lib, name)


def test_host_argument_checks_without_gpu(lib):
    h = ctypes.c_void_p(1234)
    # negative size, bad enums, null out-pointer: rejected before any CUDA call
    assert lib.sptrsv_analyze(-1, 0, None, None, None, 0, 0, 0, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.sptrsv_analyze(4, 4, None, None, None, 0, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.sptrsv_analyze(0, 0, None, None, None, 7, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.sptrsv_analyze(0, 0, None, None, None, 0, 3, 0, None, ctypes.byref(h)) == 1
    assert lib.sptrsv_analyze(0, 0, None, None, None, 0, 0, 2, None, None) == 1
    # sizes past SPTRSV_MAX_SIZE (2^31 - 256): a lane's cursor over a row's
    # entries runs up to 128 entries past the row's end and must stay an int
    big = 2 ** 31 - 255
    m = re.search(r"#define\s+SPTRSV_MAX_SIZE\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == big - 1
    from paper_1710_04985_gb300 import _lib
    assert _lib.MAX_SIZE == big - 1
    p8 = ctypes.c_void_p(8)
    assert lib.sptrsv_analyze(1, big, p8, p8, p8, 0, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.sptrsv_analyze(big, 1, p8, p8, p8, 0, 0, 1, None, ctypes.byref(h)) == 1
    assert h.value is None
    row = ctypes.c_int(7)
    assert lib.sptrsv_solve_noalloc(1, big, p8, p8, p8, 0, 0, 0, p8, p8, None,
                                    ctypes.byref(row)) == 1
    # a non-unit matrix with no stored entry has a zero pivot in row 0
    assert lib.sptrsv_analyze(3, 0, ctypes.c_void_p(8), None, None, 0, 0, 0, None,
                              ctypes.byref(h)) == 3
    assert lib.sptrsv_last_error_row() == 0
    # calls on a null plan
    assert lib.sptrsv_solve(None, None, None, 1, 1, 1, None) == 1
    assert lib.sptrsv_solve_transpose(None, None, None, 1, 1, 0, None) == 1
    assert lib.sptrsv_set_tuning(None, 4, 256, 0) == 1
    assert lib.sptrsv_set_spin_limit(None, 10) == 1
    assert lib.sptrsv_free(None) == 1
    assert lib.sptrsv_reanalyze(None, 0, 1, None) == 1
    assert lib.sptrsv_set_partition(None, 0, 1) == 1
    assert lib.sptrsv_set_algo_tuning(None, 1, 4, 256, 0) == 1
    v = ctypes.c_int()
    assert lib.sptrsv_get_partition(None, ctypes.byref(v), ctypes.byref(v)) == 1
    assert lib.sptrsv_last_launch_count(None) == 0


def test_status_strings(lib):
    names = [lib.sptrsv_status_string(i).decode() for i in range(9)]
    assert names == ["SPTRSV_OK", "SPTRSV_ERR_INVALID_ARG", "SPTRSV_ERR_STRUCTURE",
                     "SPTRSV_ERR_ZERO_PIVOT", "SPTRSV_ERR_CUDA", "SPTRSV_ERR_OOM",
                     "SPTRSV_ERR_TIMEOUT", "SPTRSV_ERR_NOT_SUPPORTED", "SPTRSV_ERR_INTERNAL"]


def test_oracle_and_cuda_path_share_no_code():
    """Neither side imports, includes or links the other."""
    pkg = os.path.join(ROOT, "paper_1710_04985_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "sptrsv_oracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1710_04985_gb300" not in text, f
            assert "#include \"" not in text, f
    import oracle
    out = subprocess.run(["nm", "-D", "--defined-only", oracle._build.library_path()],
                         capture_output=True, text=True, check=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert syms and all(s.startswith("oracle_") for s in syms)


def test_operation_entry_points_cite_the_passage_they_implement():
    """Every call that computes something names the part of the paper that
    defines it (section, algorithm, equation or table) in its comment."""
    text = open(HEADER).read()
    comments = {m.group(2): m.group(1) for m in re.finditer(
        r"/\*((?:(?!\*/).)*)\*/\s*SPTRSV_API[^;]*?\b(sptrsv_\w+)\s*\(", text, re.S)}
    ops = ("sptrsv_analyze", "sptrsv_reanalyze", "sptrsv_solve", "sptrsv_solve_transpose",
           "sptrsv_prepare_transpose", "sptrsv_prepare", "sptrsv_grad_vals", "sptrsv_residual",
           "sptrsv_solve_refined", "sptrsv_levels", "sptrsv_transpose_pattern",
           "sptrsv_partition_info", "sptrsv_solve_noalloc")
    for name in ops:
        assert name in comments, name
        assert re.search(r"\b(Sec\.|Alg\.|eq\.|Table)", comments[name]), name
