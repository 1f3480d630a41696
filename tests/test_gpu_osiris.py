"""The parameter set of the paper's OSIRIS comparison (Sec. III; single bunch, 200 x 500 cells,
9 macroparticles per cell, 2.5e6 beam macroparticles) at full size through the C ABI: the
first pipelined beam steps against the FP64 oracle in both precisions, and the whole 1.4 m
run.  The paper prints only figures for this run, so the run itself is checked for what
they show: the driver loses energy to the wake while some of its electrons gain."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KP_INV_M = 0.367e-3  # c / omega_p at n_p = 2.1e14 cm^-3 (Sec. III)


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _gpu_steps(wk, cfg, prec, nsteps):
    import torch
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    with wk.Simulations([cfg], prec) as s:
        tb = torch.from_numpy(nm_b).cuda()
        torch.cuda.synchronize()
        wk.wake_load_plasma(s.h, 0, None if nm_p is None else torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, tb)
        d0 = s.diagnostics()[0]
        wk.wake_step(s.h, nsteps)
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        xyz, lost = s.beam(0)
        out = f, xyz.cpu().numpy(), lost.cpu().numpy(), d0, s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    return out


def _oracle_steps(cfg, nsteps):
    pl = oracle.plasma_init(cfg, synth.plasma_normals(cfg))
    bm = oracle.beam_init(cfg, synth.beam_normals(cfg))
    ref = oracle.run(cfg, pl, bm, nsteps)
    return ref, bm


def test_osiris_set_fp64_steps_match_oracle(wk):
    cfg = synth.config_osiris()
    f, xyz, lost, _, _ = _gpu_steps(wk, cfg, wk.WAKE_FP64, 2)
    ref, bm = _oracle_steps(cfg, 2)
    assert np.array_equal(lost, bm["lost"])
    keep = bm["lost"] == 0
    for row, key in enumerate(("x", "y", "xi", "ux", "uy", "uz")):
        a, b = xyz[row][keep], bm[key][keep]
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1.0), key
    scale = np.abs(ref["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        assert np.abs(f[k] - ref[k]).max() <= 1e-8 * scale, k


def test_osiris_set_mixed_steps_match_oracle(wk):
    """Mixed form, the blowout tolerances: peak on-axis |E_z| within 1%, the driver's mean
    energy change within 0.5%.  (In this cold plasma the node-wise E_z error reaches ~2% of
    the peak at the spike where the plasma electrons recross the axis; the spike's position
    is sensitive to rounding.)"""
    cfg = synth.config_osiris()
    f, _, lost, d0, d1 = _gpu_steps(wk, cfg, wk.WAKE_MIXED, 2)
    ref, bm = _oracle_steps(cfg, 2)
    dr = oracle.diagnostics(cfg, bm)
    assert np.array_equal(lost, bm["lost"])
    pk_ref = np.abs(ref["ez"][:, 0]).max()
    assert abs(np.abs(f["ez"][:, 0]).max() - pk_ref) <= 0.01 * pk_ref
    loss, loss_ref = d1[4] - d0[4], dr[4] - d0[4]
    assert loss_ref < 0.0
    assert abs(loss - loss_ref) <= 0.005 * abs(loss_ref), (loss, loss_ref)


def test_osiris_set_whole_run(wk):
    """1.4 m (Sec. III) in pipelined steps of 5 k_p^-1: the driver's mean energy falls while
    its most energetic electrons end above the initial energy (Fig. 2, bottom)."""
    cfg = synth.config_osiris()
    nsteps = int(round(1.4 / KP_INV_M / cfg.ds))
    f, xyz, lost, d0, d1 = _gpu_steps(wk, cfg, wk.WAKE_MIXED, nsteps)
    g = np.sqrt(1.0 + xyz[3] ** 2 + xyz[4] ** 2 + xyz[5] ** 2)[lost == 0]
    assert d1[4] < d0[4] - 1.0  # mean loss (units of m c^2)
    assert g.max() > cfg.gamma_b + 1.0  # some electrons gained
    assert np.isfinite(f["ez"]).all()
