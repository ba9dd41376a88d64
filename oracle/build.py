"""Build the CPU oracle (test infrastructure) into oracle/libspegg_oracle.so.

Plain gcc, no optimisation flags that change floating-point semantics:
-ffp-contract=off keeps every double operation a separately rounded IEEE
operation (no fused multiply-add), on x86-64 and on aarch64 alike.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "spegg_oracle.c"), os.path.join(HERE, "spatial_oracle.c")]
LIB = os.path.join(HERE, "libspegg_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in SRCS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
