"""The committed ncu summaries: short text files whose commands are safe to
re-run as written (clocks left alone, full-set captures bounded to one kernel
and a few launches), and every summary the benchmark reads exists and parses.
"""
import os
import re

import pytest

import bench

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def _files():
    return sorted(os.listdir(PROFILES))


def _ncu_commands(text):
    """Each ncu command of the file's code blocks, continuation lines joined."""
    cmds, cur, fenced = [], None, False
    for line in text.splitlines():
        if line.strip().startswith("```"):
            fenced = not fenced
            continue
        if not fenced:
            continue
        s = line.strip()
        if cur is not None:
            cur += " " + s.rstrip("\\").strip()
            if not s.endswith("\\"):
                cmds.append(cur)
                cur = None
            continue
        if "ncu " in s:
            s = s[s.index("ncu "):]
            if s.endswith("\\"):
                cur = s.rstrip("\\").strip()
            else:
                cmds.append(s)
    return cmds


def test_profiles_are_short_text_summaries():
    files = _files()
    assert files, "no ncu summaries committed"
    for f in files:
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(PROFILES, f)) < 16 * 1024, f
        assert not re.search(r"r\d\d|round", f), f     # named for kernel and workload


def test_every_ncu_command_leaves_the_clocks_alone_and_full_sets_stay_small():
    seen = 0
    for f in _files():
        for cmd in _ncu_commands(open(os.path.join(PROFILES, f)).read()):
            seen += 1
            assert "--clock-control none" in cmd, (f, cmd)
            if "--set full" in cmd:
                assert re.search(r"-k\s+\S+", cmd), (f, cmd)
                m = re.search(r"-c\s+(\d+)", cmd)
                assert m and int(m.group(1)) <= 3, (f, cmd)
    assert seen >= len(_files())


def test_the_benchmarks_profiles_exist_and_parse():
    for algo, (kernel, src, prof) in bench.KERNELS.items():
        if prof is None:
            assert bench.ncu_traffic("0" * 12, algo) is None
            continue
        text = open(os.path.join(PROFILES, prof)).read()
        assert kernel in text, (algo, prof)
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*\(kernel source sha\s*"
                      r"([0-9a-f]{12})\)", text)
        assert m, prof
        # read back only for the source it was taken on
        assert bench.ncu_traffic(m.group(2), algo) == pytest.approx(float(m.group(1)))
        assert bench.ncu_traffic("f" * 12, algo) is None
