"""Failure detection without a GPU fault: the pipelined steps' bounded waits run out and
report WAKE_ETIMEOUT while the context stays usable; host-injected NaN inputs raise
WAKE_ENUMERIC; a beam placed wholly outside the box is all lost.  Nothing here can fault or
hang the device: every wait polls a bounded number of times, and every index a non-finite
value produces is clamped to the grid."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _run_steps(wk, cfg, prec, nsteps):
    import torch
    with wk.Simulations([cfg], prec) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(synth.plasma_normals(cfg)).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(synth.beam_normals(cfg)).cuda())
        wk.wake_step(s.h, nsteps)
        st = s.status(0)
        xyz, lost = s.beam(0)
        return st, xyz.cpu().numpy(), lost.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pipeline_wait_runs_out_and_context_stays_usable(wk, prec, monkeypatch):
    """WAKE_SPIN_LIMIT=0 (read by wake_init) lets each wait of a pipelined step poll once: a
    step that finds the step before it not yet far enough along gives up, sets the timeout
    status and leaves; so do the steps after it.  A fresh handle with the default limit then
    runs the same steps."""
    p = wk.WAKE_FP64 if prec == "fp64" else wk.WAKE_MIXED
    cfg = synth.config_blowout(n_beam=1 << 14, nr=64, nxi=256)
    monkeypatch.setenv("WAKE_SPIN_LIMIT", "0")
    st, _, _ = _run_steps(wk, cfg, p, 6)
    assert st == wk.WAKE_ETIMEOUT
    assert "wait" in wk.wake_last_error()
    monkeypatch.delenv("WAKE_SPIN_LIMIT")
    st, xyz, lost = _run_steps(wk, cfg, p, 6)
    assert st == wk.WAKE_OK, wk.wake_last_error()
    assert np.isfinite(xyz[:, lost == 0]).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_plasma_normals_raise_numeric(wk, prec):
    import torch
    p = wk.WAKE_FP64 if prec == "fp64" else wk.WAKE_MIXED
    cfg = synth.config_blowout(n_beam=0, nr=64, nxi=128)
    nm = synth.plasma_normals(cfg).copy()
    nm[10:14] = np.nan  # two mirrored pairs of one cell
    with wk.Simulations([cfg], p) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm).cuda())
        wk.wake_plasma_march(s.h)
        assert s.status(0) == wk.WAKE_ENUMERIC
    # a clean handle afterwards marches normally
    with wk.Simulations([cfg], p) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(synth.plasma_normals(cfg)).cuda())
        wk.wake_plasma_march(s.h)
        assert s.status(0) == wk.WAKE_OK


def test_beam_outside_the_box_is_all_lost(wk):
    """Particles set beyond the box (xi >= L, xi < 0 or r >= R) start lost, are neither
    deposited nor pushed, and leave the plasma response that of no driver at all: the
    oracle's driverless march of the same warm plasma (its sampling noise only)."""
    import torch

    import oracle
    cfg = synth.config_blowout(n_beam=4096, nr=32, nxi=64)
    n = cfg.n_beam
    xyz = np.zeros((6, n))
    xyz[2] = np.where(np.arange(n) % 3 == 0, cfg.ximax + 0.5, np.where(np.arange(n) % 3 == 1, -0.5, 1.0))
    xyz[0] = np.where(np.arange(n) % 3 == 2, cfg.rmax + 0.1, 0.0)
    xyz[5] = cfg.gamma_b
    nm = synth.plasma_normals(cfg)
    ref = oracle.march(cfg, oracle.plasma_init(cfg, nm), np.zeros((cfg.nxi + 1, cfg.nr + 1)))
    for prec, tol in ((wk.WAKE_FP64, 1e-12), (wk.WAKE_MIXED, 1e-5)):
        want = xyz.copy()
        if prec == wk.WAKE_MIXED:  # x, y, u_x, u_y are kept in FP32 by the mixed form
            want[[0, 1, 3, 4]] = want[[0, 1, 3, 4]].astype(np.float32)
        with wk.Simulations([cfg], prec) as s:
            wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm).cuda())
            wk.wake_set_beam(s.h, 0, torch.from_numpy(xyz).cuda())
            wk.wake_step(s.h, 2)
            out, lost = s.beam(0)
            assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
            assert (lost.cpu().numpy() == 1).all()
            np.testing.assert_array_equal(out.cpu().numpy(), want)
            d = s.diagnostics()[0]
            assert d[0] == 0 and d[3] == 0
            assert float(s.nb(0).abs().max()) == 0.0
            f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        for k in ("psi", "ez", "er", "bth"):
            assert np.abs(f[k] - ref[k]).max() <= tol, (prec, k)
