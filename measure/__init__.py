"""Measurement tools used by bench.py and the ncu recipes under profiles/.

Not part of the solver: ``probe.cu`` (an FMA-throughput probe, built into
``measure/lib/libiga_measure.so``) states the FP64/FP32 ALU ceilings beside the
nominal figures, and ``profile_cases`` launches small, self-contained kernel
sequences for Nsight Compute captures.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_lib = None


def lib():
    """Load the measurement library (once); build() must have run."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: run measure.build.build()")
        L = C.CDLL(_build.LIB)
        L.measure_probe_fma.restype = C.c_int
        L.measure_probe_fma.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
        _lib = L
    return _lib
