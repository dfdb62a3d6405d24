"""Build of the CUDA library (in-tree, sm_103a only).

``python -m paper_2103_08253_gb300.build`` compiles ``csrc/dmn.cu`` (the DMN
update: C ABI and the thread-per-point kernels), ``csrc/dmn_warp.cu`` (its warp
organisation for small calls), ``csrc/fe.cu`` (the hexahedral FE operator and
PCG) and ``csrc/peak.cu`` (the measured FMA peaks of the rooflines) with nvcc, in
parallel, and links them into ``_build/libdmn.so`` next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "csrc", "dmn.cu"), os.path.join(HERE, "csrc", "dmn_warp.cu"),
           os.path.join(HERE, "csrc", "fe.cu"), os.path.join(HERE, "csrc", "peak.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "dmn_device.cuh"), os.path.join(HERE, "csrc", "dmn_launch.cuh"),
                  os.path.join(ROOT, "include", "dmn.h"),
                  os.path.join(ROOT, "include", "fe.h"), os.path.join(ROOT, "include", "dmn_peak.h")]
LIB = os.path.join(HERE, "_build", "libdmn.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build the DMN library")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the shared library if any source is newer than it; returns its path."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(os.path.dirname(LIB), os.path.basename(src) + ".tmp%d.o" % os.getpid())
        cmd = [nvcc(), *flags, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), flush=True)
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    rcs = [p.wait() for p in procs]
    try:
        for src, rc in zip(SOURCES, rcs):
            if rc != 0:
                raise subprocess.CalledProcessError(rc, "nvcc " + src)
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
