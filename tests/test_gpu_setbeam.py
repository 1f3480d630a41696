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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pushes_through_uniform_fields_accumulate_xi_and_uz(wk, prec):
    """Many pushes through bound uniform fields (Eqs. 8-11).  With E = B = 0 the beam streams:
    u stays as it was and xi grows by dt (1 + u_perp^2) / (gamma (gamma + u_z)) a step, ~3e-9,
    far below the FP32 spacing of xi ~ 5 (5e-7).  With a uniform E_z = c every step kicks u_z
    by -dt c = -5e-3, about one FP32 spacing of u_z = 4e4.  After 2000 steps both sums hold to
    2e-5 of their change in either form: the mixed form's xi and u_z must be kept wider than
    FP32 (an FP32 sum would leave xi where it was and miss u_z by ~1)."""
    import torch
    cfg = synth.config_blowout(n_beam=4096, nr=64, nxi=128)
    precision = wk.WAKE_FP64 if prec == "fp64" else wk.WAKE_MIXED
    fdt = torch.float64 if prec == "fp64" else torch.float32
    n, nsteps, c = cfg.n_beam, 2000, 1e-3
    rng = np.random.default_rng(11)
    xyz0 = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2.0, cfg.ximax - 2.0, n),
                     rng.normal(0, 0.3, n), rng.normal(0, 0.3, n), cfg.gamma_b + rng.uniform(-100, 100, n)])
    if prec == "mixed":  # the state the mixed form holds: x, y, u_x, u_y in FP32, xi and u_z
        for row in (0, 1, 3, 4):  # as float-float pairs
            xyz0[row] = xyz0[row].astype(np.float32).astype(np.float64)
        for row in (2, 5):
            hi = xyz0[row].astype(np.float32).astype(np.float64)
            xyz0[row] = hi + (xyz0[row] - hi).astype(np.float32).astype(np.float64)
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
    out = {}
    for ez in (0.0, c):
        with wk.Simulations([cfg], precision) as s:
            own = [torch.zeros((cfg.nxi + 1, cfg.nr + 1), dtype=fdt, device="cuda") for _ in range(4)]
            wk.wake_bind_fields(s.h, 0, *own)
            wk.wake_load_plasma(s.h, 0, nm_p)
            wk.wake_set_beam(s.h, 0, torch.from_numpy(xyz0).cuda())
            wk.wake_beam_deposit(s.h)
            wk.wake_plasma_march(s.h)
            for t in own:  # the march wrote its wake; replace it by the uniform fields
                t.zero_()
            own[1].fill_(ez)
            wk.wake_beam_push_steps(s.h, nsteps)
            xyz, lost = s.beam(0)
            assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
            assert int(lost.sum()) == 0
            out[ez] = xyz.cpu().numpy()
    free, kicked = out[0.0], out[c]
    # free streaming: the momenta do not change at all, xi by nsteps slips
    assert np.array_equal(free[3:6], xyz0[3:6])
    up2 = xyz0[3] ** 2 + xyz0[4] ** 2
    gam = np.sqrt(1 + up2 + xyz0[5] ** 2)
    dxi = nsteps * cfg.ds * (1 + up2) / (gam * (gam + xyz0[5]))
    assert np.abs((free[2] - xyz0[2]) - dxi).max() <= 2e-5 * dxi.min()
    # the uniform E_z: u_z falls by nsteps dt c
    duz = -nsteps * cfg.ds * c
    assert np.abs((kicked[5] - xyz0[5]) - duz).max() <= 2e-5 * abs(duz)
    assert np.array_equal(kicked[3:5], xyz0[3:5])
