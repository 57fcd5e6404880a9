"""Measured FMA rates of the FP64 and FP32 pipes (the tracer's roofline denominators).

The tracer is bound by arithmetic on the FP64 pipe (FP64 path) or the FP32
pipe (mixed and double-float paths).  ``measure`` runs the FMA-chain probe of
``csrc/tt_peaks.cu`` (built into ``_build/libtt_peaks.so``) on the current
device and returns the achieved rate in TFLOP/s, 2 flops per FMA.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import _build

_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_build.build_peaks())
            L.tt_fma_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.tt_fma_peak.restype = C.c_int
            _lib = L
    return _lib


def run(fp64: bool, iters: int, blocks_per_sm: int = 4):
    """One probe launch: (TFLOP/s, ms)."""
    t, ms = C.c_double(), C.c_double()
    st = lib().tt_fma_peak(1 if fp64 else 0, blocks_per_sm, iters, C.byref(t), C.byref(ms))
    if st != 0:
        raise RuntimeError("tt_fma_peak failed with status %d" % st)
    return t.value, ms.value


def measure(fp64: bool, seconds: float = 0.5, reps: int = 3) -> dict:
    """Best of ``reps`` launches sized to about ``seconds`` each."""
    iters = 200 if fp64 else 2000
    tf, ms = run(fp64, iters)
    iters = max(1, int(iters * seconds * 1e3 / max(ms, 1e-3)))
    best = (0.0, 0.0)
    for _ in range(reps):
        tf, ms = run(fp64, iters)
        if tf > best[0]:
            best = (tf, ms)
    return {"tflops": best[0], "ms_per_launch": best[1], "iters": iters, "reps": reps,
            "pipe": "fp64" if fp64 else "fp32"}
