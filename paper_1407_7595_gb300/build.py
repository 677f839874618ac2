"""Build libmem.so (the CUDA product library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into a shared
library next to this file. No CMake; one -gencode target.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmem.so")
PEAK_SRC = os.path.join(HERE, "peaks", "alu_peak.cu")
PEAK_LIB = os.path.join(HERE, "libpeak.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Division and square root at 2 ulp (MUFU-based) and flush-to-zero: the FP32 integrand
# error budget (1e-5 per point) is dominated by conditioning, not by these roundings.
# sinf/atan2f/expf keep their accurate library forms (no -use_fast_math).
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-prec-div=false", "-prec-sqrt=false", "-ftz=true",
         "-Xptxas", "-warn-spills"]


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _newest_input():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "mem.h"))
    return max(os.path.getmtime(f) for f in files)


def build_peak(force=False, verbose=False):
    """The ALU microbenchmark library (FP32/FP64/MUFU peaks for the roofline); not
    part of the integrator."""
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= os.path.getmtime(PEAK_SRC):
        return PEAK_LIB
    tmp = PEAK_LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                           "-cudart", "static", PEAK_SRC, "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def build(force=False, verbose=False):
    peak = None
    if force or not os.path.exists(PEAK_LIB):
        peak = subprocess.Popen([sys.executable, "-c", "import sys; sys.path.insert(0, %r); "
                                 "import build as B; B.build_peak(force=True)" % HERE])
    try:
        return _build_lib(force, verbose)
    finally:
        if peak is not None and peak.wait() != 0:
            raise RuntimeError("nvcc failed for peaks/alu_peak.cu")


def _build_lib(force=False, verbose=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [NVCC] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out = p.communicate()[0].decode(errors="replace")
        if p.returncode != 0:
            failed.append(src)
            sys.stderr.write(out)
        elif verbose and out.strip():
            sys.stderr.write(out)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    # static CUDA runtime (nvcc default): the library needs only the driver at run time
    subprocess.run([NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
