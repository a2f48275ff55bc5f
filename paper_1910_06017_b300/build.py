"""Builds libomt.so, the CUDA library of the tracking hot path, in-tree.

nvcc compiles every csrc/*.cu for sm_103a (B300) only; the objects are
linked into paper_1910_06017_b300/libomt.so.  probe/fma_peak.cu becomes
probe/libomt_probe.so, the benchmark's FP32 throughput probe.  Usage:
    python -m paper_1910_06017_b300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libomt.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    subprocess.check_call(cmd)
    return obj


PROBE_SRC = os.path.join(PKG, "probe", "fma_peak.cu")
PROBE_LIB = os.path.join(PKG, "probe", "libomt_probe.so")


def build_probe(force: bool = False) -> str:
    """libomt_probe.so: the FP32 multiply-add throughput probe the benchmark
    uses as the LK kernel's roofline (not part of the tracking library)."""
    if force or not os.path.exists(PROBE_LIB) or os.path.getmtime(PROBE_LIB) < os.path.getmtime(PROBE_SRC):
        tmp = PROBE_LIB + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, *ARCH, *FLAGS, "-shared", "-o", tmp, PROBE_SRC, "-lcudart"])
        os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    build_probe(force)
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
