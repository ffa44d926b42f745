"""Build the CUDA library ``_build/libsptrsv.so`` (sm_103a only) in-tree.

nvcc compiles each translation unit in parallel, then links a shared library
that exports the C ABI of ``include/sptrsv.h``.  A second small library,
``_build/libsptrsv_cusparse_ref.so``, wraps cuSPARSE SpSV for the benchmark's
comparison column; the solver never links it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["api.cu", "analysis.cu", "solve_self.cu", "solve_level.cu", "solve_mrhs.cu", "aux.cu",
           "solve_tiled.cu", "solve_chain.cu", "noalloc.cu", "permute.cu",
           "solve_column.cu", "kahn.cu", "solve_blocked.cu", "solve_parts.cu", "refine.cu"]
CUSPARSE_SOURCES = ["cusparse_ref.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def library_path() -> str:
    return os.path.join(OUT, "libsptrsv.so")


def cusparse_ref_path() -> str:
    return os.path.join(OUT, "libsptrsv_cusparse_ref.so")


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hdrs + [os.path.join(INCLUDE, "sptrsv.h")]


def _compile(nvcc, src, obj, extra, verbose):
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
           "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def _link(nvcc, objs, out, libs, verbose):
    libdir = _cuda_lib_dir(nvcc)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-L", libdir, "-Xlinker", "-rpath", "-Xlinker", libdir, *libs]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(out)} failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> str:
    """Compile both libraries if any source is newer than them."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    deps = _deps()
    jobs = []
    for group, out, libs in ((SOURCES, library_path(), []),
                             (CUSPARSE_SOURCES, cusparse_ref_path(), ["-lcusparse"])):
        srcs = [os.path.join(CSRC, s) for s in group]
        if force or ptxas_info or _stale(out, srcs + deps):
            jobs.append((srcs, out, libs))
    if not jobs:
        return library_path()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        futs = {}
        for srcs, out, libs in jobs:
            for s in srcs:
                obj = os.path.join(OUT, os.path.basename(s) + ".o")
                futs[ex.submit(_compile, nvcc, s, obj, extra, verbose)] = obj
        for f in cf.as_completed(futs):
            msg = f.result()
            if ptxas_info and msg:
                print(msg)
    for srcs, out, libs in jobs:
        objs = [os.path.join(OUT, os.path.basename(s) + ".o") for s in srcs]
        _link(nvcc, objs, out, libs, verbose)
    return library_path()


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv))
