"""Launch-group run schedule (host logic, no GPU): every member's tiles formed
exactly once, the prefetch shares numbered per member, each block's runs in
member order and every block's work within a set-up or two per round of the
average.  The check is a small C++ program linked against the built library."""
import os
import shutil
import subprocess

import pytest

from paper_1603_09255_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def test_schedule_covers_balances_and_orders(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    pkg_build.build()
    lib = pkg_build.OUT_DIR
    exe = str(tmp_path / "schedule_check")
    cmd = ["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1603_09255_gb300", "csrc"), "-I", cuda_include(),
           os.path.join(ROOT, "tests", "schedule_check.cpp"), "-L", lib, "-lspegg_gb300",
           "-Wl,-rpath," + lib, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    ratios = [float(line.split()[5]) for line in r.stdout.splitlines() if len(line.split()) == 6]
    # groups with a piece of 8 tiles or more per block (the library's pieces
    # hold 8192 offspring, tiles at most 1024): within 10 % of a perfect split
    busy = [float(l.split()[5]) for l in r.stdout.splitlines()
            if len(l.split()) == 6 and int(l.split()[2]) >= 8
            and int(l.split()[3]) >= int(l.split()[1]) * int(l.split()[2])]
    assert len(ratios) == 300 and busy and max(busy) < 1.10, max(busy)
