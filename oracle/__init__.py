"""FP64 CPU oracle for the quasi-static r-xi wake march and the beam-driver push.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg
are the only callers.  The library path never imports this package, and this package never
imports the library.  ``wake_oracle.c`` holds the arithmetic (plain C, one thread, FP64,
compiled without FMA contraction so that it gives the same numbers on x86-64 and AArch64);
this module compiles it with gcc on first use and marshals NumPy arrays through ctypes.

Each wrapped routine names the passage of the paper (arXiv:1411.3246) it follows; the C
source states the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wake_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENUMERIC, EESCAPE = 0, -1, -2, -4, -6

# node-array slots written by solve_slice (see the SL_* enum in wake_oracle.c)
SLOTS = ["psi", "dpsi", "ez", "bth", "er", "rho", "jz", "chi", "T", "Q", "kcell"]


class OrcParams(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nxi", C.c_int32), ("ppc", C.c_int32), ("pad0", C.c_int32),
                ("rmax", C.c_double), ("ximax", C.c_double), ("u_th", C.c_double),
                ("n_d", C.c_double), ("n_w", C.c_double), ("sigma_r", C.c_double),
                ("sigma_zd", C.c_double), ("sigma_zw", C.c_double), ("xi_d", C.c_double),
                ("xi_w", C.c_double), ("gamma_b", C.c_double), ("eps_n", C.c_double),
                ("ds", C.c_double), ("n_beam", C.c_int64), ("n_drive", C.c_int64),
                ("geometry", C.c_int32), ("pad1", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            d, i32, i64 = C.c_double, C.c_int, C.c_int64
            pd, pu8, pp = P(d), P(C.c_uint8), P(OrcParams)
            L.orc_gamma_uz.argtypes = [d, d, pd, pd]
            L.orc_plasma_init.argtypes = [pp, pd, pd, pd, pd, pd, pd]
            L.orc_plasma_init.restype = i32
            L.orc_nb_eq12.argtypes = [pp, d, d]
            L.orc_nb_eq12.restype = d
            L.orc_nb_analytic.argtypes = [pp, pd]
            L.orc_tridiag.argtypes = [i32, pd, pd, pd, pd, pd]
            L.orc_tridiag.restype = i32
            L.orc_solve_slice.argtypes = [pp, i32, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd]
            L.orc_solve_slice.restype = i32
            L.orc_deposit_charge.argtypes = [pp, i32, pd, pd, pd]
            L.orc_march.argtypes = [pp, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd]
            L.orc_march.restype = i32
            L.orc_beam_weights.argtypes = [pp, pd, pd]
            L.orc_beam_init.argtypes = [pp, pd, pd, pd, pd, pd, pd, pd, pu8]
            L.orc_beam_deposit.argtypes = [pp, pd, pd, pd, pu8, pd]
            L.orc_beam_push.argtypes = [pp, pd, pd, pd, pd, pd, pd, pu8, pd, pd, pd]
            L.orc_diagnostics.argtypes = [pp, pd, pd, pd, pu8, pd]
            L.orc_run.argtypes = [pp, i32, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pu8,
                                  pd, pd, pd, pd]
            L.orc_run.restype = i32
            L.orc_run_w.argtypes = [pp, i32, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pu8,
                                    pd, pd, pd, pd, pd]
            L.orc_run_w.restype = i32
            L.orc_witness_obs.argtypes = [pp, pd, pd, pd, pu8, pd, pd]
            pi32 = P(C.c_int)
            L.orc_march_trap.argtypes = [pp, pd, pd, pd, pd, pd, pd, d, pd, pd, pd, pd, pd, pd, i32, pi32]
            L.orc_march_trap.restype = i32
            L.orc_beam_deposit_wt.argtypes = [pp, i64, pd, pd, pd, pu8, pd, pd]
            pi64 = P(C.c_int64)
            L.orc_run_trap.argtypes = [pp, i32, pd, pd, pd, pd, pd, d, i64, pi64, pd, pd, pd, pd, pd, pd, pu8,
                                       pd, pu8, pi64, pd, pd, pd, pd]
            L.orc_run_trap.restype = i32
            L.orc_beam_deposit_w.argtypes = [pp, pd, pd, pd, pu8, pd, pd]
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(C.POINTER(C.c_double))
    if a.dtype == np.uint8:
        return a.ctypes.data_as(C.POINTER(C.c_uint8))
    raise TypeError(a.dtype)


def params(cfg) -> OrcParams:
    """OrcParams from a synth.WakeConfig (or any object with the same attributes)."""
    return OrcParams(cfg.nr, cfg.nxi, cfg.ppc, 0, cfg.rmax, cfg.ximax, cfg.u_th, cfg.n_d,
                     cfg.n_w, cfg.sigma_r, cfg.sigma_zd, cfg.sigma_zw, cfg.xi_d, cfg.xi_w,
                     cfg.gamma_b, cfg.eps_n, cfg.ds, cfg.n_beam, cfg.n_drive,
                     int(getattr(cfg, "geometry", 0)), 0)


class OracleError(RuntimeError):
    pass


def _check(status, what):
    if status != OK:
        raise OracleError(f"{what}: oracle status {status}")


def gamma_uz(uperp2: float, Gam: float):
    """Eqs. 2-3: gamma and u_z of a plasma electron from u_perp^2 and Gamma = Gamma0 + psi."""
    g, u = C.c_double(), C.c_double()
    lib().orc_gamma_uz(uperp2, Gam, C.byref(g), C.byref(u))
    return g.value, u.value


def plasma_init(cfg, normals):
    """Initial plasma slice (Sec. II.A, warm Maxwellian momenta): dict of r0, ur0, l, G0, w."""
    p = params(cfg)
    n = cfg.nr * cfg.ppc
    out = {k: np.zeros(n) for k in ("r0", "ur0", "l", "G0", "w")}
    nm = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    _check(lib().orc_plasma_init(C.byref(p), _p(nm), _p(out["r0"]), _p(out["ur0"]), _p(out["l"]),
                                 _p(out["G0"]), _p(out["w"])), "plasma_init")
    return out


def nb_analytic(cfg):
    """Eq. 12 two-bunch density on the (nxi+1) x (nr+1) nodes."""
    p = params(cfg)
    nb = np.zeros((cfg.nxi + 1, cfg.nr + 1))
    lib().orc_nb_analytic(C.byref(p), _p(nb))
    return nb


def nb_eq12(cfg, r, xi):
    p = params(cfg)
    return lib().orc_nb_eq12(C.byref(p), float(r), float(xi))


def tridiag(a, b, c, d):
    """Thomas algorithm: a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = np.zeros_like(d)
    _check(lib().orc_tridiag(len(d), _p(a), _p(b), _p(c), _p(d), _p(x)), "tridiag")
    return x


def deposit_charge(cfg, r, w):
    p = params(cfg)
    rho = np.zeros(cfg.nr + 1)
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    lib().orc_deposit_charge(C.byref(p), len(r), _p(r), _p(w), _p(rho))
    return rho


def solve_slice(cfg, r, ur, ut, G0, w, rho0, nb_slice):
    """One slice: deposits and the radial field solves of Eqs. 6-7.  Returns a dict of the
    node arrays in SLOTS plus per-particle Gamma and the Cartesian radial force."""
    p = params(cfg)
    n1 = cfg.nr + 1
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (r, ur, ut, G0, w, rho0, nb_slice)]
    out = np.zeros(len(SLOTS) * n1)
    np_ = len(arrs[0])
    G = np.zeros(max(np_, 1))
    F = np.zeros(max(np_, 1))
    _check(lib().orc_solve_slice(C.byref(p), np_, *[_p(a) for a in arrs], _p(out), _p(G), _p(F)),
           "solve_slice")
    res = {k: out[i * n1:(i + 1) * n1].copy() for i, k in enumerate(SLOTS)}
    res["kcell"] = res["kcell"][:cfg.nr]
    res["Gamma"] = G[:np_]
    res["Fc"] = F[:np_]
    return res


def march(cfg, plasma, nb, traj=False):
    """The xi-march for a frozen beam density nb: returns psi, ez, er, bth on the
    (nxi+1) x (nr+1) nodes (and the ring trajectories r, u_r, Gamma if traj)."""
    p = params(cfg)
    shape = (cfg.nxi + 1, cfg.nr + 1)
    out = {k: np.zeros(shape) for k in ("psi", "ez", "er", "bth")}
    nb = np.ascontiguousarray(nb, dtype=np.float64)
    tr = np.zeros((cfg.nxi + 1, 3, cfg.nr * cfg.ppc)) if traj else None
    _check(lib().orc_march(C.byref(p), _p(plasma["r0"]), _p(plasma["ur0"]), _p(plasma["l"]),
                           _p(plasma["G0"]), _p(plasma["w"]), _p(nb), _p(out["psi"]), _p(out["ez"]),
                           _p(out["er"]), _p(out["bth"]), _p(tr)), "march")
    if traj:
        out["traj"] = tr
    return out


def beam_weights(cfg):
    p = params(cfg)
    wd, ww = C.c_double(), C.c_double()
    lib().orc_beam_weights(C.byref(p), C.byref(wd), C.byref(ww))
    return wd.value, ww.value


def beam_init(cfg, normals):
    """Beam state from the normals (Eq. 12 bunches): dict x, y, xi, ux, uy, uz, lost."""
    p = params(cfg)
    n = cfg.n_beam
    b = {k: np.zeros(n) for k in ("x", "y", "xi", "ux", "uy", "uz")}
    b["lost"] = np.zeros(n, dtype=np.uint8)
    nm = np.ascontiguousarray(normals, dtype=np.float64)
    lib().orc_beam_init(C.byref(p), _p(nm), *[_p(b[k]) for k in ("x", "y", "xi", "ux", "uy", "uz", "lost")])
    return b


def beam_deposit(cfg, beam, wmul=None):
    """Beam density on the nodes; wmul: optional per-particle charge multipliers."""
    p = params(cfg)
    nb = np.zeros((cfg.nxi + 1, cfg.nr + 1))
    wm = None if wmul is None else np.ascontiguousarray(wmul, dtype=np.float64)
    lib().orc_beam_deposit_w(C.byref(p), _p(beam["x"]), _p(beam["y"]), _p(beam["xi"]), _p(beam["lost"]), _p(wm),
                             _p(nb))
    return nb


def beam_push(cfg, beam, fields):
    """One Boris step of Eqs. 8-11 in place."""
    p = params(cfg)
    f = {k: np.ascontiguousarray(fields[k], dtype=np.float64) for k in ("er", "ez", "bth")}
    lib().orc_beam_push(C.byref(p), *[_p(beam[k]) for k in ("x", "y", "xi", "ux", "uy", "uz", "lost")],
                        _p(f["er"]), _p(f["ez"]), _p(f["bth"]))


def diagnostics(cfg, beam):
    """[witness count, witness mean gamma, witness rms gamma, drive count, drive mean gamma]."""
    p = params(cfg)
    out = np.zeros(5)
    lib().orc_diagnostics(C.byref(p), _p(beam["ux"]), _p(beam["uy"]), _p(beam["uz"]), _p(beam["lost"]), _p(out))
    return out


def run(cfg, plasma, beam, nsteps, wmul=None):
    """nsteps beam steps (deposit, march, push) in place on beam; returns the last fields.
    wmul: optional per-particle charge multipliers (a witness current profile)."""
    p = params(cfg)
    shape = (cfg.nxi + 1, cfg.nr + 1)
    out = {k: np.zeros(shape) for k in ("psi", "ez", "er", "bth")}
    wm = None if wmul is None else np.ascontiguousarray(wmul, dtype=np.float64)
    _check(lib().orc_run_w(C.byref(p), nsteps, _p(plasma["r0"]), _p(plasma["ur0"]), _p(plasma["l"]),
                           _p(plasma["G0"]), _p(plasma["w"]),
                           *[_p(beam[k]) for k in ("x", "y", "xi", "ux", "uy", "uz", "lost")], _p(wm),
                           _p(out["psi"]), _p(out["ez"]), _p(out["er"]), _p(out["bth"])), "run")
    return out


def witness_obs(cfg, beam, wmul=None):
    """Charge-weighted witness mean energy gain and rms energy spread (Sec. IV)."""
    p = params(cfg)
    out = np.zeros(2)
    wm = None if wmul is None else np.ascontiguousarray(wmul, dtype=np.float64)
    lib().orc_witness_obs(C.byref(p), _p(beam["ux"]), _p(beam["uy"]), _p(beam["uz"]), _p(beam["lost"]),
                          _p(wm), _p(out))
    return out


def witness_objective(cfg, theta, profile, plasma_normals, beam_normals, nsteps):
    """The witness observables after nsteps beam steps as a function of the parameters the
    adjoint differentiates: theta = (n_w, xi_w - xi_d, sigma_zd, u_th) and the witness current
    profile (multipliers of the witness charge in len(profile) bins of xi_w +- 3 sigma_zw,
    by each particle's xi draw).  Returns (mean gain, rms spread)."""
    import copy
    c = copy.copy(cfg)
    c.n_w, c.xi_w, c.sigma_zd, c.u_th = float(theta[0]), c.xi_d + float(theta[1]), float(theta[2]), float(theta[3])
    pl = plasma_init(c, plasma_normals)
    bm = beam_init(c, beam_normals)
    wm = np.ones(c.n_beam)
    nb = len(profile)
    if nb > 0:
        z = beam_normals[4, c.n_drive:]
        b = np.clip(np.floor((z + 3.0) * nb / 6.0).astype(np.int64), 0, nb - 1)
        wm[c.n_drive:] = np.asarray(profile, dtype=np.float64)[b]
    run(c, pl, bm, nsteps, wm)
    return witness_obs(c, bm, wm)


def march_trap(cfg, plasma, nb, gamma_t, traj=False):
    """The xi-march with trapping (Sec. I: plasma particles past a threshold become beam
    particles): rings whose Gamma falls below gamma_t leave the plasma.  Returns the fields (and
    trajectories if traj) and "trap", an (n, 7) array of (ring, slice, r, u_r, u_theta, Gamma,
    weight) per promotion."""
    p = params(cfg)
    shape = (cfg.nxi + 1, cfg.nr + 1)
    out = {k: np.zeros(shape) for k in ("psi", "ez", "er", "bth")}
    nb = np.ascontiguousarray(nb, dtype=np.float64)
    n = cfg.nr * cfg.ppc
    tr = np.zeros((cfg.nxi + 1, 3, n)) if traj else None
    trap = np.zeros((n, 7))
    nt = C.c_int(0)
    _check(lib().orc_march_trap(C.byref(p), _p(plasma["r0"]), _p(plasma["ur0"]), _p(plasma["l"]), _p(plasma["G0"]),
                                _p(plasma["w"]), _p(nb), float(gamma_t), _p(out["psi"]), _p(out["ez"]), _p(out["er"]),
                                _p(out["bth"]), _p(tr), _p(trap), n, C.byref(nt)), "march_trap")
    out["trap"] = trap[:min(nt.value, n)].copy()
    out["n_promoted"] = nt.value
    if traj:
        out["traj"] = tr
    return out


def run_trap(cfg, plasma, beam, nsteps, gamma_t, cap):
    """nsteps beam steps with trapping (orc_run_trap): beam (oracle.beam_init's dict) grows to at
    most cap particles.  Returns (fields of the last march, beam dict of cap entries with "wt"
    weights and "tag" 0 drive / 1 witness / 2 promoted, particles in use, dropped promotions)."""
    p = params(cfg)
    n0 = cfg.n_beam
    b = {k: np.zeros(cap) for k in ("x", "y", "xi", "ux", "uy", "uz", "wt")}
    b["lost"] = np.ones(cap, dtype=np.uint8)
    b["tag"] = np.zeros(cap, dtype=np.uint8)
    for k in ("x", "y", "xi", "ux", "uy", "uz"):
        b[k][:n0] = beam[k]
    b["lost"][:n0] = beam["lost"]
    wd, ww = beam_weights(cfg)
    b["wt"][:n0] = np.where(np.arange(n0) < cfg.n_drive, wd, ww)
    b["tag"][:n0] = np.where(np.arange(n0) < cfg.n_drive, 0, 1)
    shape = (cfg.nxi + 1, cfg.nr + 1)
    out = {k: np.zeros(shape) for k in ("psi", "ez", "er", "bth")}
    n_cur, dropped = C.c_int64(n0), C.c_int64(0)
    _check(lib().orc_run_trap(C.byref(p), nsteps, _p(plasma["r0"]), _p(plasma["ur0"]), _p(plasma["l"]),
                              _p(plasma["G0"]), _p(plasma["w"]), float(gamma_t), cap, C.byref(n_cur),
                              *[_p(b[k]) for k in ("x", "y", "xi", "ux", "uy", "uz", "lost", "wt", "tag")],
                              C.byref(dropped), _p(out["psi"]), _p(out["ez"]), _p(out["er"]), _p(out["bth"])), "run_trap")
    return out, b, n_cur.value, dropped.value
