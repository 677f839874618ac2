"""Measured ALU peaks of the current GPU (FP32 FFMA, FP64 DFMA, MUFU EX2/RSQ).

Loads libpeak.so (built from peaks/alu_peak.cu by build.py) and times full-occupancy
grids of independent dependent chains of one operation each, with CUDA events on
the library's own stream. These rates are the denominators of the integrand
kernels' roofline fractions (FP32 for the single-lepton processes, FP64 for the
dilepton neutrino solution). Nothing here changes a clock or power setting.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
PEAK_LIB = os.path.join(HERE, "libpeak.so")
OPS = {"fp32_ffma": 0, "fp64_dfma": 1, "mufu_ex2": 2, "mufu_rsq": 3}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(PEAK_LIB):
            raise RuntimeError(f"{PEAK_LIB} is missing: run __graft_entry__.build() first")
        _lib = C.CDLL(PEAK_LIB)
        _lib.alu_peak_run.restype = C.c_int
        _lib.alu_peak_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
    return _lib


def run(op, iters, blocks_per_sm=8, reps=5):
    """(operations per second, best launch ms) of one operation's chains."""
    r, ms = C.c_double(), C.c_double()
    rc = lib().alu_peak_run(OPS[op], blocks_per_sm, iters, reps, C.byref(r), C.byref(ms))
    if rc != 0:
        raise RuntimeError(f"alu_peak_run({op}) failed with CUDA error {rc}")
    return r.value, ms.value


def measure(target_ms=40.0):
    """All four rates; each op's loop count is scaled from a short calibration launch
    so that one launch takes about target_ms. Returns TFLOP/s for the FMA pipes
    (an FMA = 2 flops) and G operations/s for MUFU."""
    out = {}
    for op in OPS:
        rate, ms = run(op, 16, reps=1)
        iters = max(16, int(16 * target_ms / max(ms, 1e-3)))
        rate, ms = run(op, iters)
        if op.startswith("fp"):
            out[op.split("_")[0] + "_tflops"] = 2.0 * rate / 1e12
        else:
            out[op + "_gops"] = rate / 1e9
        out[op + "_launch_ms"] = ms
    return out
