"""GB300 (sm_103a) quasi-static wake march and beam push (arXiv:1411.3246, WAKE).

The compute path is libwake.so (CUDA kernels behind the C ABI of include/wake.h);
``paper_1411_3246_gb300.wake`` is its thin ctypes binding and ``paper_1411_3246_gb300.build``
compiles it.  There is no CPU fallback: the binding raises if the library is missing.
"""
__all__ = ["wake", "build"]
