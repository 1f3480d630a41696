"""Slab geometry (x, xi) on the GPU against the FP64 oracle's slab reading, through the C ABI.

The same tolerances as the cylindrical parity tests: FP64 to ~1e-10 of peak (linear) and
1e-8 (warm blowout); the mixed form within 1e-5 of peak in the linear case and, in blowout,
the peak on-axis E_z within 1% and the witness energy gain within 0.5%.  Plus the pipelined
steps (one launch of many steps) against the separate calls, the trajectory dump, and the
refusals (trapping, the adjoint) that the slab reading leaves out.
"""
import ctypes as C

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


def _march(wk, cfg, prec, normals=None):
    import torch
    with wk.Simulations([cfg], prec) as s:
        nm = None if normals is None else torch.from_numpy(normals).cuda()
        wk.wake_load_plasma(s.h, 0, nm)
        wk.wake_plasma_march(s.h)
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    return f


def _oracle_march(cfg):
    nm = synth.plasma_normals(cfg)
    return oracle.march(cfg, oracle.plasma_init(cfg, nm), oracle.nb_analytic(cfg)), nm


@pytest.mark.parametrize("nr,nxi", [(128, 256), (100, 77), (2, 8), (512, 64)])
def test_slab_linear_march_fp64_matches_oracle(wk, nr, nxi):
    cfg = synth.config_slab_linear(nr=nr, nxi=nxi)
    ref, _ = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_FP64)
    scale = np.abs(ref["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        assert np.abs(f[k] - ref[k]).max() <= 1e-10 * scale, k
    # the slab wake, not the cylindrical one
    cyl, _ = _oracle_march(synth.config_linear(nr=nr, nxi=nxi))
    assert np.abs(cyl["psi"] - f["psi"]).max() > 1e-3 * np.abs(f["psi"]).max()


def test_slab_linear_march_mixed_within_1e5_of_peak(wk):
    cfg = synth.config_slab_linear()
    ref, _ = _oracle_march(cfg)
    for prec in (wk.WAKE_MIXED, wk.WAKE_MIXED64):
        f = _march(wk, cfg, prec)
        scale = np.abs(ref["ez"]).max()
        errs = {k: np.abs(f[k] - ref[k]).max() / scale for k in ("psi", "ez", "er", "bth")}
        assert max(errs.values()) <= 1e-5, (prec, errs)


@pytest.mark.parametrize("nr,nxi", [(64, 256), (512, 2048)])
def test_slab_blowout_warm_march_fp64_matches_oracle(wk, nr, nxi):
    cfg = synth.config_slab_blowout(n_beam=0, nr=nr, nxi=nxi)
    cfg.n_beam = 0
    ref, nm = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_FP64, nm)
    scale = np.abs(ref["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        err = np.abs(f[k] - ref[k]).max() / scale
        assert err <= 1e-8, (k, err)


def test_slab_blowout_warm_march_mixed_peak_ez(wk):
    cfg = synth.config_slab_blowout(n_beam=0)
    cfg.n_beam = 0
    ref, nm = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_MIXED, nm)
    peak_ref = np.abs(ref["ez"][:, 0]).max()
    assert abs(np.abs(f["ez"][:, 0]).max() - peak_ref) <= 0.01 * peak_ref
    k = int(round(cfg.xi_w / cfg.ximax * cfg.nxi))
    assert abs(f["ez"][k, 0] - ref["ez"][k, 0]) <= 0.01 * peak_ref


def _beam_case(n_beam, nr, nxi):
    cfg = synth.config_slab_blowout(n_beam=n_beam, nr=nr, nxi=nxi)
    return cfg, synth.plasma_normals(cfg), synth.beam_normals(cfg)


def test_slab_sheet_beam_deposit_fp64_matches_oracle(wk):
    import torch
    cfg, nm_p, nm_b = _beam_case(1 << 16, 64, 128)
    bm = oracle.beam_init(cfg, nm_b)
    ref = oracle.beam_deposit(cfg, bm)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_beam_deposit(s.h)
        nb = s.nb(0).cpu().numpy()
        xyz, lost = s.beam(0)
    xyz = xyz.cpu().numpy()
    assert np.all(xyz[1] == 0.0) and np.all(xyz[4] == 0.0)  # y = u_y = 0
    assert np.array_equal(lost.cpu().numpy(), bm["lost"])
    assert np.abs(nb - ref).max() <= 1e-12 * np.abs(ref).max()
    # the handle-free deposit folds the same sheet beam
    out = torch.zeros((cfg.nxi + 1, cfg.nr + 1), dtype=torch.float64, device="cuda")
    wk.wake_beam_deposit_noalloc(wk.params_of(cfg, wk.WAKE_FP64), torch.from_numpy(np.stack(
        [bm["x"], np.full_like(bm["x"], 5.0), bm["xi"], bm["ux"], bm["uy"], bm["uz"]])).cuda(),
        torch.from_numpy(bm["lost"]).cuda(), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_slab_beam_steps_fp64_match_oracle(wk):
    import torch
    cfg, nm_p, nm_b = _beam_case(1 << 14, 64, 256)
    pl, bm = oracle.plasma_init(cfg, nm_p), oracle.beam_init(cfg, nm_b)
    ref = oracle.run(cfg, pl, bm, 3)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, 3)
        assert wk.wake_step_kernel_ms(s.h) > 0.0  # the pipelined launch ran
        xyz, lost = s.beam(0)
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        diag = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    xyz = xyz.cpu().numpy()
    assert np.array_equal(lost.cpu().numpy(), bm["lost"])
    keep = bm["lost"] == 0
    for row, key in enumerate(("x", "y", "xi", "ux", "uy", "uz")):
        a, b = xyz[row][keep], bm[key][keep]
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1.0), key
    scale = np.abs(ref["ez"]).max()
    assert np.abs(f["ez"] - ref["ez"]).max() <= 1e-8 * scale
    d_ref = oracle.diagnostics(cfg, bm)
    assert diag[0] == d_ref[0] and diag[3] == d_ref[3]
    np.testing.assert_allclose(diag[1], d_ref[1], rtol=1e-12)


def test_slab_pipelined_mixed_full_size_against_oracle(wk):
    """The blowout box in slab geometry at the benchmark's size (512 x 2048, 2^20 particles),
    three pipelined steps in the mixed form against the oracle's: peak on-axis E_z within 1%,
    witness mean energy gain within 0.5%, the same surviving counts."""
    import torch
    cfg = synth.config_slab_blowout()
    nsteps = 3
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    pl, bm = oracle.plasma_init(cfg, nm_p), oracle.beam_init(cfg, nm_b)
    d0 = oracle.diagnostics(cfg, bm)
    ref = oracle.run(cfg, pl, bm, nsteps)
    d_ref = oracle.diagnostics(cfg, bm)
    with wk.Simulations([cfg], wk.WAKE_MIXED) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, nsteps)
        assert wk.wake_step_kernel_ms(s.h) > 0.0
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        d = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    pk_ref = np.abs(ref["ez"][:, 0]).max()
    print(f"slab: peak E_z {np.abs(f['ez'][:, 0]).max():.6f} vs {pk_ref:.6f}; gain {d[1] - d0[1]:.5f} vs "
          f"{d_ref[1] - d0[1]:.5f}")
    assert abs(np.abs(f["ez"][:, 0]).max() - pk_ref) <= 0.01 * pk_ref
    assert d[0] == d_ref[0] and d[3] == d_ref[3]
    gain, gain_ref = d[1] - d0[1], d_ref[1] - d0[1]
    assert abs(gain_ref) > 0.1
    assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref)


def test_slab_trajectory_dump_fp64_matches_oracle(wk):
    import torch
    cfg = synth.config_slab_blowout(n_beam=0, nr=64, nxi=256)
    cfg.n_beam = 0
    nm = synth.plasma_normals(cfg)
    ref = oracle.march(cfg, oracle.plasma_init(cfg, nm), oracle.nb_analytic(cfg), traj=True)["traj"]
    every = 4
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm).cuda())
        n = cfg.nr * cfg.ppc
        tr = torch.zeros(((cfg.nxi // every + 1) * 3 * n,), dtype=torch.float64, device="cuda")
        wk.wake_plasma_march_traj(s.h, 0, every, tr)
        got = tr.cpu().numpy().reshape(-1, 3, n)
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    want = ref[::every]
    assert np.abs(got - want).max() <= 1e-9 * max(np.abs(want).max(), 1.0)


def test_slab_refuses_trapping_and_the_adjoint(wk):
    cfg = synth.config_slab_blowout(n_beam=1024, nr=32, nxi=64)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        with pytest.raises(wk.WakeError) as e:
            wk.wake_set_trapping(s.h, 0, 0.5, 16)
        assert e.value.code == wk.WAKE_EINVAL
    p = wk.params_of(cfg, wk.WAKE_FP64)
    a = C.c_void_p()
    assert wk.lib().wake_adjoint_init(C.byref(p), 2, 0, None, C.byref(a)) == wk.WAKE_EINVAL
    assert not a.value


def test_bound_fields_and_frozen_wake_pushes(wk):
    """wake_bind_fields: the march writes straight into caller-owned grids (the library's own
    march to rounding) and the push reads them there; wake_beam_push_steps(n) equals n pushes."""
    import torch
    for geometry in (0, 1):
        cfg = (synth.config_slab_blowout if geometry else synth.config_blowout)(n_beam=1 << 12, nr=64, nxi=128)
        nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
        nm_b = torch.from_numpy(synth.beam_normals(cfg)).cuda()
        got = []
        for bind in (False, True):
            with wk.Simulations([cfg], wk.WAKE_FP64) as s:
                own = [torch.full((cfg.nxi + 1, cfg.nr + 1), float("nan"), dtype=torch.float64, device="cuda")
                       for _ in range(4)]
                if bind:
                    wk.wake_bind_fields(s.h, 0, *own)
                wk.wake_load_plasma(s.h, 0, nm_p)
                wk.wake_load_beam(s.h, 0, nm_b)
                wk.wake_beam_deposit(s.h)
                wk.wake_plasma_march(s.h)
                if bind:
                    f = {k: v.cpu().numpy() for k, v in zip(("psi", "ez", "er", "bth"), own)}
                    with pytest.raises(wk.WakeError):  # after a march: refused
                        wk.wake_bind_fields(s.h, 0, *own)
                else:
                    f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
                wk.wake_beam_push_steps(s.h, 3)
                xyz = s.beam(0)[0].cpu().numpy()
                assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
            got.append((f, xyz))
        # the same march (the FP64 deposit sums differ only in the order of their atomics)
        for k in ("psi", "ez", "er", "bth"):
            a, b = got[0][0][k], got[1][0][k]
            assert np.isfinite(b).all() and np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), k
        assert np.abs(got[0][1] - got[1][1]).max() <= 1e-10 * np.abs(got[0][1]).max()
        # three frozen-wake pushes = three separate pushes
        with wk.Simulations([cfg], wk.WAKE_FP64) as s:
            wk.wake_load_plasma(s.h, 0, nm_p)
            wk.wake_load_beam(s.h, 0, nm_b)
            wk.wake_beam_deposit(s.h)
            wk.wake_plasma_march(s.h)
            for _ in range(3):
                wk.wake_beam_push(s.h)
            xyz3 = s.beam(0)[0].cpu().numpy()
        assert np.abs(xyz3 - got[0][1]).max() <= 1e-10 * np.abs(got[0][1]).max()
