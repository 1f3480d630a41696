"""Long oracle runs in worker processes, for the GPU parity tests at full size.

The workers are started with spawn (never forked from a process that has touched the GPU),
so that the FP64 oracle's minutes-long runs overlap the GPU work and one another.  Each job
rebuilds its inputs from the configuration's seeds, as the GPU side does.
"""
from __future__ import annotations

import multiprocessing as mp

import numpy as np


def pool(procs):
    return mp.get_context("spawn").Pool(procs)


def run_steps(cfg, nsteps):
    """The workload from its initial state through nsteps beam steps: the diagnostics before
    and after, the last march's fields on the axis and at every node (E_z), and the beam."""
    import oracle
    import synth
    pl = oracle.plasma_init(cfg, synth.plasma_normals(cfg))
    bm = oracle.beam_init(cfg, synth.beam_normals(cfg))
    d0 = oracle.diagnostics(cfg, bm)
    f = oracle.run(cfg, pl, bm, nsteps)
    return {"d0": d0, "d": oracle.diagnostics(cfg, bm), "ez": f["ez"].astype(np.float32), "ez_axis": f["ez"][:, 0].copy(),
            "lost": bm["lost"], "uz": bm["uz"]}


def witness_objective(cfg, theta, profile, nsteps):
    """The adjoint form's observables (mean gain, rms spread) after nsteps steps."""
    import oracle
    import synth
    return oracle.witness_objective(cfg, np.asarray(theta, dtype=np.float64), np.asarray(profile, dtype=np.float64),
                                    synth.plasma_normals(cfg), synth.beam_normals(cfg), nsteps)
