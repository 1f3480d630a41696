"""wake_set_beam: a beam given by the caller (state, per-particle weights, witness tags)
through the C ABI - a saved state continues exactly, and per-particle weights deposit as the
FP64 oracle's deposit with the same charges."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _case():
    return synth.config_blowout(n_beam=1 << 14, nr=64, nxi=256)


def test_saved_state_continues_like_the_original_run(wk):
    import torch
    cfg = _case()
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).cuda()
    with wk.Simulations([cfg], wk.WAKE_FP64) as a:
        wk.wake_load_plasma(a.h, 0, nm_p)
        wk.wake_load_beam(a.h, 0, nm_b)
        wk.wake_step(a.h, 2)
        xyz, lost = a.beam(0)
        wk.wake_step(a.h, 3)
        ref_xyz, ref_lost = a.beam(0)
        ref_ez = a.fields(0)["ez"].cpu().numpy()
        assert a.status(0) == wk.WAKE_OK, wk.wake_last_error()
    xyz = xyz.clone()
    xyz[2][lost.bool()] = -1.0  # keep lost particles lost: move them out of the box
    tag = (torch.arange(cfg.n_beam, device="cuda") >= cfg.n_drive).to(torch.uint8)
    with wk.Simulations([cfg], wk.WAKE_FP64) as b:
        wk.wake_load_plasma(b.h, 0, nm_p)
        wk.wake_set_beam(b.h, 0, xyz, None, tag)
        wk.wake_step(b.h, 3)
        got_xyz, got_lost = b.beam(0)
        got_ez = b.fields(0)["ez"].cpu().numpy()
        assert b.status(0) == wk.WAKE_OK, wk.wake_last_error()
    assert np.array_equal(got_lost.cpu().numpy(), ref_lost.cpu().numpy())
    keep = ref_lost.cpu().numpy() == 0
    g, r = got_xyz.cpu().numpy()[:, keep], ref_xyz.cpu().numpy()[:, keep]
    assert np.abs(g - r).max() <= 1e-10 * np.abs(r).max()
    assert np.abs(got_ez - ref_ez).max() <= 1e-10 * np.abs(ref_ez).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_per_particle_weights_deposit_as_the_oracle(wk, prec):
    import torch
    cfg = _case()
    nm_b = synth.beam_normals(cfg)
    bm = oracle.beam_init(cfg, nm_b)
    rng = np.random.default_rng(7)
    wmul = rng.uniform(0.5, 1.5, cfg.n_beam)
    wd, ww = oracle.beam_weights(cfg)
    w = np.where(np.arange(cfg.n_beam) < cfg.n_drive, wd, ww) * wmul
    ref = oracle.beam_deposit(cfg, bm, wmul)
    xyz = np.stack([bm["x"], bm["y"], bm["xi"], bm["ux"], bm["uy"], bm["uz"]])
    p = wk.WAKE_FP64 if prec == "fp64" else wk.WAKE_MIXED
    with wk.Simulations([cfg], p) as s:
        wk.wake_set_beam(s.h, 0, torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda(), None)
        wk.wake_beam_deposit(s.h)
        nb = s.nb(0).cpu().numpy()
        _, lost = s.beam(0)
        assert np.array_equal(lost.cpu().numpy(), bm["lost"])
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(nb - ref).max() <= tol * np.abs(ref).max()
