"""CUDA path vs the FP64 oracle, through the C ABI, on the same seeded inputs.

FP64 form: every field node and beam coordinate agrees to ~1e-10 relative.  Mixed form
(FP32 ring arithmetic and fields): fields within 1e-5 of peak |E_z| in the linear case; in
blowout, the peak on-axis E_z within 1% and the witness mean energy gain and spread within
0.5%.
"""
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


@pytest.mark.parametrize("nr,nxi", [(128, 256), (100, 77), (2, 8), (1024, 64)])
def test_linear_march_fp64_matches_oracle(wk, nr, nxi):
    cfg = synth.config_linear(nr=nr, nxi=nxi)
    ref, _ = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_FP64)
    scale = np.abs(ref["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        assert np.abs(f[k] - ref[k]).max() <= 1e-10 * scale, k


def test_linear_march_mixed_within_1e5_of_peak(wk):
    cfg = synth.config_linear()
    ref, _ = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_MIXED)
    scale = np.abs(ref["ez"]).max()
    errs = {k: np.abs(f[k] - ref[k]).max() / scale for k in ("psi", "ez", "er", "bth")}
    assert max(errs.values()) <= 1e-5, errs


@pytest.mark.parametrize("nr,nxi", [(64, 256), (512, 2048)])
def test_blowout_warm_march_fp64_matches_oracle(wk, nr, nxi):
    cfg = synth.config_blowout(n_beam=0, nr=nr, nxi=nxi)
    cfg.n_beam = 0
    ref, nm = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_FP64, nm)
    scale = np.abs(ref["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        err = np.abs(f[k] - ref[k]).max() / scale
        assert err <= 1e-8, (k, err)


def test_blowout_warm_march_mixed_peak_ez(wk):
    cfg = synth.config_blowout(n_beam=0)
    cfg.n_beam = 0
    ref, nm = _oracle_march(cfg)
    f = _march(wk, cfg, wk.WAKE_MIXED, nm)
    peak_ref = np.abs(ref["ez"][:, 0]).max()
    peak = np.abs(f["ez"][:, 0]).max()
    assert abs(peak - peak_ref) <= 0.01 * peak_ref
    # the accelerating field at the witness centre
    k = int(round(cfg.xi_w / cfg.ximax * cfg.nxi))
    assert abs(f["ez"][k, 0] - ref["ez"][k, 0]) <= 0.01 * peak_ref


def _beam_case(n_beam, nr, nxi):
    cfg = synth.config_blowout(n_beam=n_beam, nr=nr, nxi=nxi)
    return cfg, synth.plasma_normals(cfg), synth.beam_normals(cfg)


def test_beam_deposit_fp64_matches_oracle(wk):
    import torch
    cfg, nm_p, nm_b = _beam_case(1 << 16, 64, 128)
    bm = oracle.beam_init(cfg, nm_b)
    ref = oracle.beam_deposit(cfg, bm)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_beam_deposit(s.h)
        nb = s.nb(0).cpu().numpy()
        xyz, lost = s.beam(0)
    assert np.array_equal(lost.cpu().numpy(), bm["lost"])
    assert np.abs(nb - ref).max() <= 1e-12 * np.abs(ref).max()


def test_beam_steps_fp64_match_oracle(wk):
    import torch
    cfg, nm_p, nm_b = _beam_case(1 << 14, 64, 256)
    pl, bm = oracle.plasma_init(cfg, nm_p), oracle.beam_init(cfg, nm_b)
    ref = oracle.run(cfg, pl, bm, 3)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, 3)
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
    np.testing.assert_allclose(diag[2], d_ref[2], rtol=1e-6, atol=1e-9)


def test_beam_steps_mixed_witness_energy(wk):
    """Mixed form over several steps: witness mean energy gain and spread within 0.5% of
    the FP64 oracle's."""
    import torch
    cfg, nm_p, nm_b = _beam_case(1 << 16, 128, 512)
    cfg.ds = 50.0  # fewer, larger steps: a measurable energy change
    pl, bm = oracle.plasma_init(cfg, nm_p), oracle.beam_init(cfg, nm_b)
    d0 = oracle.diagnostics(cfg, bm)
    oracle.run(cfg, pl, bm, 4)
    d_ref = oracle.diagnostics(cfg, bm)
    with wk.Simulations([cfg], wk.WAKE_MIXED) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, 4)
        diag = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    gain_ref, gain = d_ref[1] - d0[1], diag[1] - d0[1]
    assert abs(gain) > 10.0
    assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref)
    assert abs(diag[2] - d_ref[2]) <= 0.005 * d_ref[2] + 1e-3


def test_batched_uneven_simulations_match_individual_oracles(wk):
    """One handle, one march launch, uneven sizes: each simulation matches its oracle."""
    import torch
    cfgs = [synth.config_linear(nr=64, nxi=128), synth.config_linear(nr=100, nxi=300, n0=0.05),
            synth.config_blowout(n_beam=0, nr=48, nxi=96)]
    cfgs[2].n_beam = 0
    refs = [_oracle_march(c) for c in cfgs]
    with wk.Simulations(cfgs, wk.WAKE_FP64) as s:
        for i, (ref, nm) in enumerate(refs):
            wk.wake_load_plasma(s.h, i, None if nm is None else torch.from_numpy(nm).cuda())
        wk.wake_plasma_march(s.h)
        for i, (ref, nm) in enumerate(refs):
            f = {k: v.cpu().numpy() for k, v in s.fields(i).items()}
            scale = np.abs(ref["ez"]).max()
            for k in ("psi", "ez", "er", "bth"):
                assert np.abs(f[k] - ref[k]).max() <= 1e-8 * scale, (i, k)
