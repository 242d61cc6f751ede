"""Build the CUDA library librich.so in-tree (sm_103a only).

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked into ``paper_2309_12496_gb300/librich.so`` with the CUDA runtime
linked statically, so the library depends only on the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librich.so")

SOURCES = ["rich_kernels.cu", "rich_capi.cu", "rich_static.cu", "rich_peaks.cu", "rich_bvh.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    p = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(p):
        return p
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librich.so")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def _flags(extra=()):
    # Plain FP32 `/` and sqrtf compile to the hardware approximations (a few
    # ulp): they only serve geometry, whose FP32 error budget they fit. Every
    # FP32 operation that decides an integer (a wavelength, a table bin, an
    # accept/reject) is written with the IEEE-rounded intrinsics (__fdiv_rn,
    # __fmul_rn, ...), which these flags do not touch.
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
                   "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC,-fvisibility=hidden", *extra]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + _headers())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link librich.so; returns its path."""
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        if force or ptxas_info or _stale(obj, src):
            extra = ["-Xptxas", "-v"] if ptxas_info and s.endswith(".cu") else []
            jobs.append([nvcc, *_flags(extra), "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            logs = list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fvisibility=hidden"])
        os.replace(tmp, LIB)
    if verbose or ptxas_info:
        for log in logs:
            sys.stdout.write(log)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
