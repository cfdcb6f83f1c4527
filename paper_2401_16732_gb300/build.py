"""Build the CUDA library in-tree: nvcc for sm_103a, one shared object.

    python -m paper_2401_16732_gb300.build
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libflashgpu.so")
PEAKS_LIB = os.path.join(PKG, "libflpeaks.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "--extended-lambda"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + [
        os.path.join(ROOT, "include", "flashgpu.h"), os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [NVCC, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + ".tmp"
    subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


def build_peaks(force: bool = False) -> str:
    """The roofline-ceiling measurements (csrc/peaks, libflpeaks.so) used by
    the throughput measurements; not part of the convolution library."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "peaks", "*.cu")))
    deps = srcs + [os.path.join(ROOT, "include", "flpeaks.h"), os.path.join(CSRC, "fl_device.cuh")]
    if not force and os.path.exists(PEAKS_LIB):
        t = os.path.getmtime(PEAKS_LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return PEAKS_LIB
    tmp = PEAKS_LIB + ".tmp"
    subprocess.check_call([NVCC, *FLAGS, "-shared", "-o", tmp, *srcs])
    os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    print(build_peaks(force="--force" in sys.argv))
