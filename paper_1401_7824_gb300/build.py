"""Build the CUDA library libisdc.so in-tree with nvcc for sm_103a.

The library is plain C ABI (include/isdc.h); nothing here links against
PyTorch.  Rebuilds when a source is newer than the library."""
from __future__ import annotations

import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libisdc.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(PKG, "csrc", "*.cuh"))) + [os.path.join(ROOT, "include", "isdc.h")]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


PROBE_LIB = os.path.join(PKG, "libisdc_probe.so")
PROBE_SRC = os.path.join(PKG, "csrc", "probe", "fp64_rate.cu")


def build_probe(force: bool = False) -> str:
    """libisdc_probe.so: the FP64 issue-rate measurement (include/isdc_probe.h)."""
    deps_p = [PROBE_SRC, os.path.join(ROOT, "include", "isdc_probe.h")]
    if not force and os.path.exists(PROBE_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(PROBE_LIB)
                                                       for d in deps_p):
        return PROBE_LIB
    tmp = f"{PROBE_LIB}.tmp{os.getpid()}"
    subprocess.check_call([nvcc(), ARCH, "-O3", "-lineinfo", "-shared", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                           "-o", tmp, PROBE_SRC])
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps()):
            return LIB
    tmp = f"{LIB}.tmp{os.getpid()}"
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
           "-o", tmp] + sources()
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_probe(force=True))
