"""Parameter studies of the paper's Sec. IV on the GPU path, through the public API.

* Temperature: the on-axis E_z behind a two-bunch driver for several plasma temperatures.
  The spike where the plasma electrons recross the axis is suppressed as T_e grows, while
  the flat region at the witness is unchanged (Sec. IV, Fig. 5).
* Grid: the spike amplitude against the slice size dxi.  In a cold plasma it keeps growing
  as dxi shrinks; in a warm one it tends to a limit (Sec. IV, Figs. 8 and 9).
* Propagation: the Table I beam carried over a distance in metres; the witness energy gain
  and spectrum (Sec. III, Fig. 3; Sec. IV, Fig. 7).
* Trajectories: the plasma electrons' paths behind the driver.  Expelled electrons fall back
  and cross the axis where the spike forms; warm electrons, with their spread of initial
  velocities, cross it over a broader region than cold ones, and a single bunch gives a
  narrower crossing than two (Sec. IV, Figs. 4 and 5).

The callers supply the simulations' parameters and random draws (the repository's `synth`
module makes the paper's workloads); this module runs them and reduces the results.

Units: the Table I plasma has n_p = 5e16 cm^-3, so k_p^-1 = 23.7 um (Sec. III), the cold
wave-breaking field m c omega_p / e is 96 sqrt(n_p[cm^-3]) V/m = 21.5 GV/m, and an energy
gamma m c^2 is 0.511e-3 gamma GeV.
"""
from __future__ import annotations

import math

import numpy as np

from . import wake

N_P_CM3 = 5.0e16
KP_INV_M = 23.7e-6
E0_GV_PER_M = 96.0 * math.sqrt(N_P_CM3) / 1.0e9
MC2_GEV = 0.511e-3


def steps_for_length(length_m: float, ds: float) -> int:
    """Beam steps of size ds (in k_p^-1) that cover length_m metres."""
    return int(round(length_m / KP_INV_M / ds))


def axis_profiles(cfgs, plasma_normals, precision=wake.WAKE_MIXED, stream=None):
    """One march per simulation (one batched handle, frozen analytic driver when a
    configuration has no beam particles).  Returns the on-axis E_z of each as a float64
    numpy array over xi_k = k dxi."""
    import torch
    with wake.Simulations(cfgs, precision, stream) as s:
        keep = [None if nm is None else torch.from_numpy(nm).cuda() for nm in plasma_normals]
        torch.cuda.synchronize()
        for i, t in enumerate(keep):
            wake.wake_load_plasma(s.h, i, t)
        wake.wake_plasma_march(s.h)
        out = [s.fields(i)["ez"][:, 0].cpu().numpy() for i in range(len(cfgs))]
        bad = [i for i in range(len(cfgs)) if s.status(i) != wake.WAKE_OK]
        del keep
    if bad:
        raise wake.WakeError(-4, f"simulations {bad} raised a numeric or escape status")
    return out


def spike_and_flat(ez_axis, cfg):
    """Accelerating spike -min E_z over the box and the flat-region field: -E_z averaged over
    the witness core |xi - xi_w| < sigma_zw / 4.  Both in units of E_0."""
    xi = np.arange(cfg.nxi + 1) * cfg.ximax / cfg.nxi
    core = np.abs(xi - cfg.xi_w) < 0.25 * cfg.sigma_zw
    return float(-ez_axis.min()), float(-ez_axis[core].mean())


def witness_energies_gev(xyz, lost, n_drive):
    """Energies (GeV) of the surviving witness particles (index >= n_drive)."""
    x = xyz[:, n_drive:]
    keep = lost[n_drive:] == 0
    ux, uy, uz = x[3][keep], x[4][keep], x[5][keep]
    return MC2_GEV * np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)


def spectrum_peak(e_gev, bin_gev=0.25):
    """Centre of the fullest bin of a histogram with bins of bin_gev."""
    lo = math.floor(e_gev.min() / bin_gev) * bin_gev
    nb = max(1, int(math.ceil((e_gev.max() - lo) / bin_gev)) + 1)
    h, edges = np.histogram(e_gev, bins=nb, range=(lo, lo + nb * bin_gev))
    k = int(np.argmax(h))
    return float(0.5 * (edges[k] + edges[k + 1]))


def propagate(cfg, plasma_normals, beam_normals, lengths_m, precision=wake.WAKE_MIXED, stream=None):
    """Carry one simulation's beam over the distances lengths_m (increasing, metres) with
    pipelined beam steps.  Returns, per distance: the steps taken, the witness mean energy
    gain and rms spread (GeV), the witness spectrum peak (GeV), the surviving witness count,
    and the kernel time of the step launches (ms)."""
    import torch
    out = []
    with wake.Simulations([cfg], precision, stream) as s:
        tp = None if plasma_normals is None else torch.from_numpy(plasma_normals).cuda()
        tb = torch.from_numpy(beam_normals).cuda()
        torch.cuda.synchronize()
        wake.wake_load_plasma(s.h, 0, tp)
        wake.wake_load_beam(s.h, 0, tb)
        e_init = MC2_GEV * cfg.gamma_b
        done, kern_ms = 0, 0.0
        for length in lengths_m:
            n = steps_for_length(length, cfg.ds) - done
            if n > 0:
                wake.wake_step(s.h, n)
                kern_ms += wake.wake_step_kernel_ms(s.h)
                done += n
            xyz, lost = s.beam(0)
            e = witness_energies_gev(xyz.cpu().numpy(), lost.cpu().numpy(), cfg.n_drive)
            if s.status(0) != wake.WAKE_OK:
                raise wake.WakeError(s.status(0), wake.wake_last_error())
            out.append({"length_m": length, "steps": done, "mean_gain_gev": float(e.mean() - e_init),
                         "rms_gev": float(e.std()), "peak_gev": spectrum_peak(e), "alive": int(e.size),
                         "kernel_ms": kern_ms})
        del tp, tb
    return out


def trajectories(cfg, plasma_normals, every=1, precision=wake.WAKE_MIXED, stream=None):
    """One march of one simulation (frozen analytic driver when it has no beam particles) with
    the ring trajectory dump.  Returns (xi, traj): xi the dump slices' positions and traj a
    float64 numpy array (len(xi), 3, nr * ppc) of each ring's r, u_r and Gamma there."""
    import torch
    nd = cfg.nxi // every + 1
    with wake.Simulations([cfg], precision, stream) as s:
        tp = None if plasma_normals is None else torch.from_numpy(plasma_normals).cuda()
        out = torch.empty((nd, 3, cfg.nr * cfg.ppc), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        wake.wake_load_plasma(s.h, 0, tp)
        wake.wake_plasma_march_traj(s.h, 0, every, out)
        st = s.status(0)
        traj = out.cpu().numpy()
        del tp
    if st != wake.WAKE_OK:
        raise wake.WakeError(st, wake.wake_last_error())
    xi = np.arange(nd) * every * cfg.ximax / cfg.nxi
    return xi, traj


def axis_crossings(r, xi, xi_after, r_cut):
    """Per ring (columns of r, a (len(xi), n_rings) array of radii along xi): the xi of its
    first approach to the axis behind xi_after, i.e. the first dump after xi_after where its
    radius has a local minimum below r_cut; NaN for a ring that has none."""
    r = np.asarray(r)
    n_d = r.shape[0]
    out = np.full(r.shape[1], np.nan)
    k = np.arange(1, n_d - 1)
    k = k[xi[k] > xi_after]
    if k.size == 0:
        return out
    mins = (r[k - 1] > r[k]) & (r[k] <= r[k + 1]) & (r[k] < r_cut)
    has = mins.any(axis=0)
    first = np.argmax(mins, axis=0)
    out[has] = xi[k[first[has]]]
    return out


def crossing_width(xi_cross, w, lo=0.1, hi=0.9):
    """Length in xi of the axis-crossing region: the range between the lo and hi quantiles of
    the rings' crossing points, each ring weighted by its charge w (rings without a crossing
    left out).  Returns (width, fraction of the charge that crossed)."""
    ok = np.isfinite(xi_cross)
    x, ww = xi_cross[ok], np.asarray(w, dtype=np.float64)[ok]
    if x.size == 0:
        return float("nan"), 0.0
    o = np.argsort(x, kind="stable")
    x, ww = x[o], ww[o]
    c = np.cumsum(ww) / ww.sum()
    q = lambda f: float(x[min(np.searchsorted(c, f), x.size - 1)])  # noqa: E731
    return q(hi) - q(lo), float(ww.sum() / np.asarray(w, dtype=np.float64).sum())
