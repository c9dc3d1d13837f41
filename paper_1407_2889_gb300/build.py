"""Build ``libpmscan.so`` in-tree for sm_103a (GB300) with nvcc.

Translation units compile in parallel; the library lands in
``paper_1407_2889_gb300/_build/libpmscan.so``. ``ptxas -v`` output
(registers, spills, shared memory) is kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpmscan.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["scan_ac.cu", "scan_ac_wide.cu", "scan_ac_wide_counts.cu", "scan_wm.cu", "scan_batch.cu", "scan_acv.cu",
              "scan_ac2.cu"]
CPP_SOURCES = ["compile.cpp", "capi.cpp", "serve.cpp"]
HEADERS = ["pm_internal.h", "scan_common.cuh", "ac_device.cuh", "ac_scan_kernel.cuh"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA 13 toolkit is required to build libpmscan")
    return p


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "pmscan.h")]
    jobs, objs = [], []
    for src in CU_SOURCES + CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if not force and not _stale(o, [s] + hdrs + [__file__]):
            continue
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + common + ["-lineinfo", "-Xptxas", "-v", "-c", s, "-o", o]
        else:
            cmd = [nvcc] + ARCH + common + ["-x", "c++", "-c", s, "-o", o]
        log = open(o + ".log", "w")
        jobs.append((src, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), log, o))
    failed = []
    for src, proc, log, o in jobs:
        rc = proc.wait()
        log.close()
        if rc != 0:
            failed.append(src)
            with open(o + ".log") as f:
                sys.stderr.write(f"---- {src} ----\n" + f.read()[-6000:])
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    with open(os.path.join(BUILD, "ptxas.log"), "w") as out:
        for src in CU_SOURCES:
            lp = os.path.join(BUILD, src + ".o.log")
            if os.path.exists(lp):
                out.write(open(lp).read())
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
