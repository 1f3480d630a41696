"""Measured FP32 and FP64 FMA throughput of the GPU (fp_peak.cu): the ALU roofline of the
xi-march.  Built beside libwake by paper_1411_3246_gb300.build."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.path.dirname(HERE), "_build", "libfppeak.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1411_3246_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.fp_peak_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_float),
                                  C.POINTER(C.c_double)]
        L.fp_peak_run.restype = C.c_int
        _lib = L
    return _lib


def fma_tflops(fp64: bool, sms: int = 152, ctas_per_sm: int = 8, iters: int = 0, stream=None):
    """TFLOP/s of the FMA kernel (FMA = 2 flop): ctas_per_sm x sms CTAs of 256 threads, each
    thread 16 independent chains of iters FMAs (default: ~0.1 s of work at the nominal rate).
    Returns (tflops, ms, flop)."""
    if iters <= 0:
        iters = 1 << 11 if fp64 else 1 << 16
    ms, flop = C.c_float(), C.c_double()
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    rc = lib().fp_peak_run(1 if fp64 else 0, sms * ctas_per_sm, iters, st, C.byref(ms), C.byref(flop))
    if rc != 0:
        raise RuntimeError(f"fp_peak_run failed: cudaError {rc}")
    return flop.value / (ms.value * 1e-3) / 1e12, ms.value, flop.value
