"""Pipelined beam steps (wake_step on one simulation with a beam) against the same steps taken
one call at a time (wake_beam_deposit, wake_plasma_march, wake_beam_push), through the C ABI.

The two paths do the same arithmetic; only the order of the atomic deposit sums differs, so
the FP64 form agrees to rounding and the mixed form to FP32 rounding amplified by the march.
"""
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


def _run(wk, cfg, prec, plan):
    """plan: list of step counts; an int n is wake_step(n), ('seq', n) is n separate steps."""
    import torch
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    with wk.Simulations([cfg], prec) as s:
        wk.wake_load_plasma(s.h, 0, None if nm_p is None else torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        for p in plan:
            if isinstance(p, tuple):
                for _ in range(p[1]):
                    wk.wake_beam_deposit(s.h)
                    wk.wake_plasma_march(s.h)
                    wk.wake_beam_push(s.h)
            else:
                wk.wake_step(s.h, p)
        xyz, lost = s.beam(0)
        out = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        out["nb"] = s.nb(0).cpu().numpy()
        out["xyz"], out["lost"] = xyz.cpu().numpy(), lost.cpu().numpy()
        out["diag"] = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    return out


def _small(n_beam=1 << 15, nr=64, nxi=256):
    cfg = synth.config_blowout(n_beam=n_beam, nr=nr, nxi=nxi)
    return cfg


def _compare_fp64(a, b, tol):
    assert np.array_equal(a["lost"], b["lost"])
    keep = a["lost"] == 0
    for row in range(6):
        x, y = a["xyz"][row][keep], b["xyz"][row][keep]
        assert np.abs(x - y).max() <= tol * max(np.abs(y).max(), 1.0), row
    for k in ("psi", "ez", "er", "bth", "nb"):
        assert np.abs(a[k] - b[k]).max() <= tol * max(np.abs(b[k]).max(), 1e-300), k


def test_pipelined_fp64_matches_sequential(wk):
    cfg = _small()
    a = _run(wk, cfg, wk.WAKE_FP64, [12])
    b = _run(wk, cfg, wk.WAKE_FP64, [("seq", 12)])
    _compare_fp64(a, b, 1e-9)


def test_pipelined_calls_in_a_row_match_sequential(wk):
    """Two wake_step calls (a re-sort between them) and a mix with separate steps."""
    cfg = _small(n_beam=1 << 14, nr=48, nxi=160)
    a = _run(wk, cfg, wk.WAKE_FP64, [5, ("seq", 2), 7])
    b = _run(wk, cfg, wk.WAKE_FP64, [("seq", 14)])
    _compare_fp64(a, b, 1e-9)


def test_pipelined_more_steps_than_one_launch(wk):
    """1100 steps of a small box: more steps than one launch holds (1024), two launches."""
    cfg = _small(n_beam=4096, nr=32, nxi=64)
    cfg.n_d = 1.0
    a = _run(wk, cfg, wk.WAKE_FP64, [1100])
    b = _run(wk, cfg, wk.WAKE_FP64, [("seq", 1100)])
    _compare_fp64(a, b, 1e-7)


def test_fast_slipping_beam_falls_back_to_separate_steps(wk):
    """gamma_b = 3: the beam slips about a cell per step, the pipelined form does not apply and
    wake_step takes the steps one at a time (same result)."""
    cfg = _small(n_beam=4096, nr=32, nxi=64)
    cfg.gamma_b, cfg.ds, cfg.n_d, cfg.n_w = 3.0, 1.0, 0.5, 0.15
    a = _run(wk, cfg, wk.WAKE_FP64, [6])
    b = _run(wk, cfg, wk.WAKE_FP64, [("seq", 6)])
    _compare_fp64(a, b, 1e-12)


def test_pipelined_mixed_matches_sequential(wk):
    cfg = _small(n_beam=1 << 16, nr=128, nxi=512)
    cfg.ds = 50.0
    a = _run(wk, cfg, wk.WAKE_MIXED, [4])
    b = _run(wk, cfg, wk.WAKE_MIXED, [("seq", 4)])
    assert np.array_equal(a["lost"], b["lost"])
    peak = np.abs(b["ez"]).max()
    assert np.abs(a["ez"] - b["ez"]).max() <= 2e-3 * peak
    da, db = a["diag"], b["diag"]
    assert da[0] == db[0] and da[3] == db[3]
    # witness mean energy gain within 0.1%
    g0 = cfg.gamma_b
    assert abs((da[1] - g0) - (db[1] - g0)) <= 1e-3 * abs(db[1] - g0)


def test_particles_slipping_several_cells_in_one_launch(wk):
    """gamma_b = 40 (linear driver): the beam slips ~1/30 cell per step, about two cells over
    60 steps of one launch; particles past their sorted cell are pushed at the cell they
    reached.  Same result as separate steps."""
    cfg = synth.config_linear(nr=64, nxi=256)
    cfg.ximax = 12.0
    cfg = synth.two_bunch(cfg, 0.3, 4.0, 4096)
    cfg.gamma_b, cfg.ds, cfg.eps_n = 40.0, 5.0, 1e-3
    a = _run(wk, cfg, wk.WAKE_FP64, [60])
    b = _run(wk, cfg, wk.WAKE_FP64, [("seq", 60)])
    _compare_fp64(a, b, 1e-8)
    nm = synth.beam_normals(cfg)
    xi0 = np.where(np.arange(cfg.n_beam) < cfg.n_drive, cfg.xi_d + cfg.sigma_zd * nm[4], cfg.xi_w + cfg.sigma_zw * nm[4])
    dxi = cfg.ximax / cfg.nxi
    live = a["lost"] == 0
    moved = np.floor(a["xyz"][2][live] / dxi) - np.floor(xi0[live] / dxi)
    assert moved.max() >= 2
