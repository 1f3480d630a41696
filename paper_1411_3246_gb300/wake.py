"""Thin ctypes binding of libwake (include/wake.h); same names as the C ABI.

Arguments are marshalled only: device arrays are torch CUDA tensors (their data_ptr() is
passed), every step of the method runs in the library's kernels.  A failing call raises
WakeError with the library's message.  There is no fallback: if libwake.so is missing this
module raises on first use.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwake.so")

WAKE_OK, WAKE_EINVAL, WAKE_ENOMEM, WAKE_ECUDA, WAKE_ENUMERIC, WAKE_ETIMEOUT, WAKE_EESCAPE, WAKE_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
WAKE_FP64, WAKE_MIXED, WAKE_MIXED64 = 0, 1, 2
WAKE_CYLINDRICAL, WAKE_SLAB = 0, 1

# every entry point the header declares
EXPORTS = ["wake_init", "wake_load_plasma", "wake_load_beam", "wake_set_beam", "wake_beam_deposit", "wake_plasma_march",
           "wake_plasma_march_traj", "wake_beam_push", "wake_beam_push_steps", "wake_bind_fields", "wake_step", "wake_tile", "wake_step_kernel_ms", "wake_get_fields", "wake_get_nb", "wake_get_beam",
           "wake_diagnostics", "wake_status", "wake_set_trapping", "wake_trapped", "wake_beam_deposit_noalloc", "wake_adjoint_init",
           "wake_adjoint_forward", "wake_adjoint_backward", "wake_adjoint_destroy", "wake_last_error", "wake_destroy"]
WAKE_NOALLOC_MAX_NODES = 524288


class wake_params(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nxi", C.c_int32), ("ppc", C.c_int32), ("precision", C.c_int32),
                ("rmax", C.c_double), ("ximax", C.c_double), ("u_th", C.c_double),
                ("n_d", C.c_double), ("n_w", C.c_double), ("sigma_r", C.c_double),
                ("sigma_zd", C.c_double), ("sigma_zw", C.c_double), ("xi_d", C.c_double),
                ("xi_w", C.c_double), ("gamma_b", C.c_double), ("eps_n", C.c_double),
                ("ds", C.c_double), ("n_beam", C.c_int64), ("n_drive", C.c_int64),
                ("geometry", C.c_int32), ("reserved", C.c_int32)]


class WakeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libwake error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libwake.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1411_3246_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, pd = C.c_void_p, C.c_int, C.POINTER(C.c_double)
        L.wake_init.argtypes = [C.POINTER(wake_params), i32, vp, C.POINTER(vp)]
        L.wake_load_plasma.argtypes = [vp, i32, vp]
        L.wake_load_beam.argtypes = [vp, i32, vp]
        L.wake_set_beam.argtypes = [vp, i32, vp, vp, vp]
        for n in ("wake_beam_deposit", "wake_plasma_march", "wake_beam_push"):
            getattr(L, n).argtypes = [vp]
        L.wake_plasma_march_traj.argtypes = [vp, i32, i32, vp]
        L.wake_beam_push_steps.argtypes = [vp, i32]
        L.wake_bind_fields.argtypes = [vp, i32, vp, vp, vp, vp]
        L.wake_step.argtypes = [vp, i32]
        L.wake_step_kernel_ms.argtypes = [vp, C.POINTER(C.c_float)]
        L.wake_tile.argtypes = [vp, i32, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.wake_get_fields.argtypes = [vp, i32, vp, vp, vp, vp]
        L.wake_get_nb.argtypes = [vp, i32, vp]
        L.wake_get_beam.argtypes = [vp, i32, vp, vp]
        L.wake_diagnostics.argtypes = [vp, pd]
        L.wake_status.argtypes = [vp, i32]
        L.wake_set_trapping.argtypes = [vp, i32, C.c_double, C.c_int64]
        L.wake_trapped.argtypes = [vp, i32, vp, vp, vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.wake_beam_deposit_noalloc.argtypes = [C.POINTER(wake_params), vp, vp, vp, vp]
        L.wake_adjoint_init.argtypes = [C.POINTER(wake_params), i32, i32, vp, C.POINTER(vp)]
        L.wake_adjoint_forward.argtypes = [vp, pd, pd, vp, vp, pd]
        L.wake_adjoint_backward.argtypes = [vp, pd, pd]
        L.wake_adjoint_destroy.argtypes = [vp]
        L.wake_adjoint_destroy.restype = None
        L.wake_last_error.restype = C.c_char_p
        L.wake_last_error.argtypes = []
        L.wake_destroy.argtypes = [vp]
        L.wake_destroy.restype = None
        for n in EXPORTS:
            if n not in ("wake_last_error", "wake_destroy", "wake_adjoint_destroy"):
                getattr(L, n).restype = i32
        _lib = L
    return _lib


def _check(rc):
    if rc != WAKE_OK:
        raise WakeError(rc, lib().wake_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device arrays must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def params_of(cfg, precision: int) -> wake_params:
    """wake_params from a parameter object with the WakeConfig attribute names."""
    return wake_params(cfg.nr, cfg.nxi, cfg.ppc, precision, cfg.rmax, cfg.ximax, cfg.u_th, cfg.n_d,
                       cfg.n_w, cfg.sigma_r, cfg.sigma_zd, cfg.sigma_zw, cfg.xi_d, cfg.xi_w,
                       cfg.gamma_b, cfg.eps_n, cfg.ds, cfg.n_beam, cfg.n_drive, int(getattr(cfg, "geometry", 0)), 0)


def wake_init(params, stream=None):
    """params: list of wake_params.  stream: a torch.cuda.Stream (None: torch's current)."""
    import torch
    arr = (wake_params * len(params))(*params)
    if stream is None:
        stream = torch.cuda.current_stream()
    h = C.c_void_p()
    _check(lib().wake_init(arr, len(params), C.c_void_p(stream.cuda_stream), C.byref(h)))
    return h


def wake_load_plasma(h, sim, normals=None):
    _check(lib().wake_load_plasma(h, sim, _ptr(normals)))


def wake_load_beam(h, sim, normals):
    _check(lib().wake_load_beam(h, sim, _ptr(normals)))


def wake_set_beam(h, sim, xyz, w=None, tag=None):
    """xyz: (6, n_beam) float64 CUDA tensor (x, y, xi, u_x, u_y, u_z); w: (n_beam,) float64 or
    None; tag: (n_beam,) uint8 or None."""
    _check(lib().wake_set_beam(h, sim, _ptr(xyz), _ptr(w), _ptr(tag)))


def wake_beam_deposit(h):
    _check(lib().wake_beam_deposit(h))


def wake_plasma_march(h):
    _check(lib().wake_plasma_march(h))


def wake_plasma_march_traj(h, sim, every, traj):
    """traj: ((nxi // every + 1), 3, nr * ppc) float64 CUDA tensor (r, u_r, Gamma per ring)."""
    _check(lib().wake_plasma_march_traj(h, sim, every, _ptr(traj)))


def wake_beam_push(h):
    _check(lib().wake_beam_push(h))


def wake_beam_push_steps(h, nsteps):
    _check(lib().wake_beam_push_steps(h, int(nsteps)))


def wake_bind_fields(h, sim, psi, ez, er, bth):
    """psi, ez, er, bth: caller-owned (nxi+1) x (nr+1) CUDA tensors of the handle's field type
    (float64 for WAKE_FP64, float32 otherwise), kept alive by the caller until wake_destroy."""
    _check(lib().wake_bind_fields(h, sim, _ptr(psi), _ptr(ez), _ptr(er), _ptr(bth)))


def wake_step(h, nsteps):
    _check(lib().wake_step(h, nsteps))


def wake_tile(h, sim):
    nt, ppt = C.c_int(), C.c_int()
    _check(lib().wake_tile(h, sim, C.byref(nt), C.byref(ppt)))
    return nt.value, ppt.value


def wake_step_kernel_ms(h):
    ms = C.c_float()
    _check(lib().wake_step_kernel_ms(h, C.byref(ms)))
    return ms.value


def wake_get_fields(h, sim, psi=None, ez=None, er=None, bth=None):
    _check(lib().wake_get_fields(h, sim, _ptr(psi), _ptr(ez), _ptr(er), _ptr(bth)))


def wake_get_nb(h, sim, nb):
    _check(lib().wake_get_nb(h, sim, _ptr(nb)))


def wake_get_beam(h, sim, xyz=None, lost=None):
    _check(lib().wake_get_beam(h, sim, _ptr(xyz), _ptr(lost)))


def wake_diagnostics(h, n_sims):
    out = (C.c_double * (5 * n_sims))()
    _check(lib().wake_diagnostics(h, out))
    return [list(out[5 * i:5 * i + 5]) for i in range(n_sims)]


def wake_beam_deposit_noalloc(params, xyz, lost, nb, stream=None):
    """params: a wake_params; xyz (6 x n_beam float64), lost (uint8) and nb ((nxi+1) x (nr+1)
    float64) CUDA tensors; stream: a torch.cuda.Stream (None: torch's current)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().wake_beam_deposit_noalloc(C.byref(params), _ptr(xyz), _ptr(lost),
                                           C.c_void_p(stream.cuda_stream), _ptr(nb)))


def wake_set_trapping(h, sim, gamma_t, capacity):
    _check(lib().wake_set_trapping(h, sim, float(gamma_t), int(capacity)))


def wake_trapped(h, sim, xyz=None, w=None, lost=None):
    """Returns (count, dropped); xyz (6, capacity), w (capacity,), lost (capacity,) float64 /
    uint8 CUDA tensors, or None, receive the promoted particles."""
    count, dropped = C.c_int64(), C.c_int64()
    _check(lib().wake_trapped(h, sim, _ptr(xyz), _ptr(w), _ptr(lost), C.byref(count), C.byref(dropped)))
    return count.value, dropped.value


def wake_status(h, sim):
    return lib().wake_status(h, sim)


def wake_last_error():
    return lib().wake_last_error().decode()


def wake_destroy(h):
    lib().wake_destroy(h)


class Simulations:
    """Convenience owner of a handle: n independent simulations on one stream."""

    def __init__(self, cfgs, precision=WAKE_MIXED, stream=None):
        import torch
        self.cfgs = list(cfgs)
        self.torch = torch
        self.stream = stream
        self.h = wake_init([params_of(c, precision) for c in self.cfgs], stream)

    def _before(self):
        """Make the handle's stream wait for torch's current stream (buffers it allocated)."""
        if self.stream is not None:
            self.stream.wait_stream(self.torch.cuda.current_stream())

    def _order(self):
        """Make torch's current stream wait for the handle's stream (outputs it wrote)."""
        if self.stream is not None:
            self.torch.cuda.current_stream().wait_stream(self.stream)

    def grid(self, sim):
        c = self.cfgs[sim]
        return self.torch.empty((c.nxi + 1, c.nr + 1), dtype=self.torch.float64, device="cuda")

    def fields(self, sim):
        out = {k: self.grid(sim) for k in ("psi", "ez", "er", "bth")}
        self._before()
        wake_get_fields(self.h, sim, out["psi"], out["ez"], out["er"], out["bth"])
        self._order()
        return out

    def nb(self, sim):
        out = self.grid(sim)
        self._before()
        wake_get_nb(self.h, sim, out)
        self._order()
        return out

    def beam(self, sim):
        c = self.cfgs[sim]
        xyz = self.torch.empty((6, c.n_beam), dtype=self.torch.float64, device="cuda")
        lost = self.torch.empty(c.n_beam, dtype=self.torch.uint8, device="cuda")
        self._before()
        wake_get_beam(self.h, sim, xyz, lost)
        self._order()
        return xyz, lost

    def diagnostics(self):
        return wake_diagnostics(self.h, len(self.cfgs))

    def status(self, sim):
        return wake_status(self.h, sim)

    def close(self):
        if self.h is not None:
            wake_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------------------
# the adjoint form
# ---------------------------------------------------------------------------------------

def _dbuf(vals):
    arr = (C.c_double * max(1, len(vals)))(*[float(v) for v in vals])
    return arr


class Adjoint:
    """Owner of a wake_adjoint handle: the witness observables (mean energy gain, rms energy
    spread) after nsteps beam steps and their gradient with respect to theta = (n_w,
    xi_w - xi_d, sigma_zd, u_th) and nbins witness-profile multipliers (include/wake.h)."""

    def __init__(self, cfg, nsteps, nbins, plasma_normals, beam_normals, stream=None):
        import torch
        self.torch = torch
        self.nbins = nbins
        self.p = params_of(cfg, WAKE_FP64)
        st = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().wake_adjoint_init(C.byref(self.p), nsteps, nbins, C.c_void_p(st.cuda_stream), C.byref(h)))
        self.h = h
        self.nm_p = plasma_normals  # device tensors kept alive for the handle's backward
        self.nm_b = beam_normals

    def forward(self, theta, profile):
        obs = (C.c_double * 2)()
        prof = _dbuf(profile)
        _check(lib().wake_adjoint_forward(self.h, _dbuf(theta), prof, _ptr(self.nm_p), _ptr(self.nm_b), obs))
        return [obs[0], obs[1]]

    def backward(self, dobs):
        g = (C.c_double * (4 + max(1, self.nbins)))()
        _check(lib().wake_adjoint_backward(self.h, _dbuf(dobs), g))
        return [g[i] for i in range(4 + self.nbins)]

    def close(self):
        if self.h is not None:
            lib().wake_adjoint_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def witness_observables(adj, theta, profile):
    """torch.autograd entry: (mean gain, rms spread) of the witness as a 2-vector, from theta
    (4,) and profile (nbins,) float64 tensors; backward runs the library's adjoint."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th, pr):
            obs = adj.forward(th.detach().cpu().tolist(), pr.detach().cpu().tolist())
            return torch.tensor(obs, dtype=torch.float64, device=th.device)

        @staticmethod
        def backward(ctx, gout):
            g = adj.backward(gout.detach().cpu().tolist())
            dev = gout.device
            return (torch.tensor(g[:4], dtype=torch.float64, device=dev),
                    torch.tensor(g[4:], dtype=torch.float64, device=dev))

    return _Fn.apply(theta, profile)
