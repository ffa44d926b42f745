"""Compile the CPU oracle (plain C) into ``oracle/_build/liboracle.so``.

Test infrastructure: building the checker is part of ``build()``, using it is
reserved to the tests, the smoke check and the benchmark's CPU baseline.
Portable flags only (the same source builds on x86_64 and aarch64).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sptrsv_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def library_path() -> str:
    return os.path.join(OUT_DIR, "liboracle.so")


def is_stale() -> bool:
    out = library_path()
    return (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(SRC)


def build(verbose: bool = False, src: str = SRC, out: str = "") -> str:
    """Compile `src` (default: the oracle) into `out` (default: the oracle
    library path)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    out = out or library_path()
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall", "-Wextra",
           src, "-o", tmp]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
