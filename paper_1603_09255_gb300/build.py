"""Build libspegg_gb300.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object, then linked into
``paper_1603_09255_gb300/_lib/libspegg_gb300.so`` against the shared CUDA
runtime.  Host code is compiled with -ffp-contract=off so the double-precision
table builders round every operation separately on x86-64 and aarch64 alike.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libspegg_gb300.so")
SOURCES = ["kernels.cu", "offspring_w1.cu", "offspring_w2.cu", "offspring_w4.cu", "offspring_w8.cu", "engine.cu",
           "population.cu", "batch.cu", "server.cu", "space.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libspegg_gb300")
    return cand


def _flags(verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "spegg.h"),
                                                                  os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f"{os.getpid()}"
    objs = [os.path.join(OUT_DIR, os.path.splitext(s)[0] + f".{tag}.o") for s in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc()] + _flags(verbose) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, zip(SOURCES, objs)))
    if verbose:
        for s, log in zip(SOURCES, logs):
            sys.stderr.write(f"== {s}\n{log}")
    tmp = LIB + f".{tag}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
                          "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        if os.path.exists(o):
            os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
