"""Fused multiply-add on numpy arrays: a * b + c with one rounding.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The oracle's fused arithmetic mode replaces each "product, then add it to a
running sum" of the rounded mode by one fused multiply-add.  numpy has no
fused multiply-add, so the element-wise operation is the C library's fma
(FP64) / fmaf (FP32) from oracle/fma.c, compiled with gcc on first use into
oracle/_build/ (or by the package build step).  Pinned by
tests/test_oracle_pins.py against exact rational arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fma.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_fma.so")

_lib = None


def build() -> str:
    """Compile oracle/fma.c into oracle/_build/liboracle_fma.so if it is
    missing or older than the source; returns the library path."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    try:
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC, "-lm"],
                       check=True, capture_output=True, text=True)
        os.replace(tmp, LIB)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_fma_f64", "oracle_fma_f32"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [ctypes.c_size_t] + [ctypes.c_void_p] * 4
        _lib = lib
    return _lib


def fma(a, b, c) -> np.ndarray:
    """a * b + c rounded once, element by element (numpy broadcasting).  The
    result type is float32 when every operand is float32, else float64."""
    dt = np.float32 if all(np.asarray(v).dtype == np.float32 for v in (a, b, c)) else np.float64
    a, b, c = np.broadcast_arrays(np.asarray(a, dtype=dt), np.asarray(b, dtype=dt), np.asarray(c, dtype=dt))
    a, b, c = (np.ascontiguousarray(v) for v in (a, b, c))
    out = np.empty(a.shape, dtype=dt)
    fn = _load().oracle_fma_f32 if dt == np.float32 else _load().oracle_fma_f64
    fn(out.size, a.ctypes.data, b.ctypes.data, c.ctypes.data, out.ctypes.data)
    return out
