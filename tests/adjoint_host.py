"""Build and call tests/adjoint_host.cpp: the library's adjoint bodies compiled for the host
(one thread), used to check the adjoint's arithmetic on machines without a GPU."""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        out = os.path.join(HERE, "_build", "adjoint_host.so")
        src = os.path.join(HERE, "adjoint_host.cpp")
        deps = [src, os.path.join(HERE, "..", "paper_1411_3246_gb300", "csrc", "adjoint_core.h")]
        if not os.path.exists(out) or any(os.path.getmtime(d) > os.path.getmtime(out) for d in deps):
            os.makedirs(os.path.dirname(out), exist_ok=True)
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-I/usr/local/cuda/include", "-o", tmp, src])
            os.replace(tmp, out)
        L = C.CDLL(out)
        pd = C.POINTER(C.c_double)
        from paper_1411_3246_gb300.wake import wake_params
        L.adj_host_gradient.argtypes = [C.POINTER(wake_params), C.c_int, C.c_int, pd, pd, pd, pd, pd, pd, pd]
        L.adj_host_gradient.restype = C.c_int
        _LIB = L
    return _LIB


def _a(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def gradient(cfg, nsteps, theta, profile, plasma_normals, beam_normals, dobs=None):
    """(obs, grad) of the host build; grad is None when dobs is None."""
    from paper_1411_3246_gb300.wake import WAKE_FP64, params_of
    p = params_of(cfg, WAKE_FP64)
    th = _a(theta)
    pr = _a(profile if len(profile) else [1.0])
    npl, nbm = _a(plasma_normals), _a(beam_normals)
    obs = np.zeros(2)
    grad = np.zeros(4 + len(profile))
    d = None if dobs is None else _a(dobs)
    rc = lib().adj_host_gradient(C.byref(p), nsteps, len(profile), th[1], pr[1], npl[1], nbm[1],
                                 None if d is None else d[1], obs.ctypes.data_as(C.POINTER(C.c_double)),
                                 grad.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 0, rc
    return obs, (grad if dobs is not None else None)
