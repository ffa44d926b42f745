"""The boundary is a C ABI: include/sptrsv.h compiles as strict C99 and as
C++, a C program links against the library, and the host-side argument
checks answer a C caller without touching a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

C_PROGRAM = r"""
#include <stdio.h>
#include "sptrsv.h"

int main(void) {
    sptrsv_plan_t plan = (sptrsv_plan_t)0;
    int fake = 0, row = 7;
    const void *p = &fake;
    int rc[5];
    /* every call below is rejected before any CUDA call */
    rc[0] = sptrsv_analyze(-1, 0, 0, 0, 0, SPTRSV_F64, SPTRSV_LOWER, SPTRSV_NON_UNIT, 0, &plan);
    rc[1] = sptrsv_analyze(1, SPTRSV_MAX_SIZE + 1, (const int *)p, (const int *)p, p, SPTRSV_F64,
                           SPTRSV_LOWER, SPTRSV_NON_UNIT, 0, &plan);
    rc[2] = sptrsv_solve(0, p, (void *)p, 1, 1, SPTRSV_ALGO_SELF, 0);
    rc[3] = sptrsv_free(0);
    rc[4] = sptrsv_solve_noalloc(1, SPTRSV_MAX_SIZE + 1, (const int *)p, (const int *)p, p,
                                 SPTRSV_F64, SPTRSV_LOWER, SPTRSV_NON_UNIT, p, (void *)p, 0, &row);
    printf("%d %d %d %d %d %s %d\n", rc[0], rc[1], rc[2], rc[3], rc[4],
           sptrsv_status_string(SPTRSV_ERR_INVALID_ARG), plan == 0);
    return 0;
}
"""


def _cc(name):
    path = shutil.which(name)
    if path is None:
        pytest.skip(f"{name} not available")
    return path


@pytest.fixture(scope="module")
def library():
    from paper_1710_04985_gb300 import build
    path = build.library_path()
    if not os.path.exists(path):
        build.build()
    return path


def test_header_is_strict_c99_and_cxx(tmp_path):
    src = tmp_path / "only_header.c"
    src.write_text('#include "sptrsv.h"\nint main(void) { return SPTRSV_OK; }\n')
    for cmd in ([_cc("gcc"), "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror"],
                [_cc("g++"), "-x", "c++", "-std=c++17", "-pedantic", "-Wall", "-Wextra",
                 "-Werror"]):
        r = subprocess.run(cmd + ["-I", INCLUDE, "-fsyntax-only", str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_c_program_links_and_gets_host_side_answers(tmp_path, library):
    from paper_1710_04985_gb300 import build
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(library)
    r = subprocess.run([_cc("gcc"), "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, str(src),
                        "-o", str(exe), "-L", libdir, "-lsptrsv"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    cuda_lib = build._cuda_lib_dir(build._nvcc())
    env["LD_LIBRARY_PATH"] = os.pathsep.join(
        [libdir, cuda_lib] + [p for p in env.get("LD_LIBRARY_PATH", "").split(os.pathsep) if p])
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["1", "1", "1", "1", "1", "SPTRSV_ERR_INVALID_ARG", "1"]
