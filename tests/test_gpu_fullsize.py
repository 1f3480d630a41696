"""Parity at the benchmark's full sizes and in the launch configuration it times: the whole
200-step run of the blowout workload (Nr=512, Nxi=2048, 2^20 beam particles) against the
oracle's (a couple of minutes of one host core, in a worker process), a few pipelined steps of
it, and three sampled simulations of the 256-simulation batched sweep run in one pipelined
batch of all 256."""
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


def test_blowout_workload_pipelined_steps_full_size(wk):
    import torch
    cfg = synth.config_blowout()  # 512 x 2048, 2^20 beam particles, as the benchmark
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
        assert wk.wake_step_kernel_ms(s.h) > 0.0  # the pipelined launch ran
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        d = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    pk_ref = np.abs(ref["ez"][:, 0]).max()
    assert abs(np.abs(f["ez"][:, 0]).max() - pk_ref) <= 0.01 * pk_ref
    assert d[0] == d_ref[0] and d[3] == d_ref[3]
    gain, gain_ref = d[1] - d0[1], d_ref[1] - d0[1]
    assert abs(gain_ref) > 1.0
    assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref), (gain, gain_ref)


def test_blowout_workload_whole_run_against_oracle(wk):
    """The benchmark's run exactly: wake_step(200) from the initial beam, mixed and FP64
    forms, against the oracle's 200 steps.  Blowout tolerances (Sec. IV results): peak
    on-axis E_z of the last march within 1%, witness mean energy gain and rms spread within
    0.5%; surviving counts equal but for particles at the box's edges.  The FP64 form agrees
    to 1e-6."""
    import torch

    import oracle_jobs
    cfg = synth.config_blowout()
    nsteps = cfg.n_steps
    assert nsteps == 200
    with oracle_jobs.pool(1) as pool:
        job = pool.apply_async(oracle_jobs.run_steps, (cfg, nsteps))
        nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
        nm_b = torch.from_numpy(synth.beam_normals(cfg)).cuda()
        got = {}
        for prec in (wk.WAKE_MIXED, wk.WAKE_FP64):
            with wk.Simulations([cfg], prec) as s:
                wk.wake_load_plasma(s.h, 0, nm_p)
                wk.wake_load_beam(s.h, 0, nm_b)
                d0 = s.diagnostics()[0]
                wk.wake_step(s.h, nsteps)
                ez = s.fields(0)["ez"].cpu().numpy()
                got[prec] = (d0, s.diagnostics()[0], ez)
                assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
        ref = job.get(timeout=1800)
    pk_ref = np.abs(ref["ez_axis"]).max()
    g_ref = ref["d"][1] - ref["d0"][1]
    s_ref = ref["d"][2]
    for prec, (tol_f, tol_g, tol_n) in ((wk.WAKE_MIXED, (1e-2, 5e-3, 1e-4)), (wk.WAKE_FP64, (1e-6, 1e-6, 0.0))):
        d0, d, ez = got[prec]
        pk = np.abs(ez[:, 0]).max()
        node = np.abs(ez - ref["ez"]).max() / pk_ref
        gain = d[1] - d0[1]
        print(f"precision {prec}: peak E_z {pk:.6f} vs {pk_ref:.6f}; node error / peak {node:.2e}; witness gain "
              f"{gain:.4f} vs {g_ref:.4f}, spread {d[2]:.4f} vs {s_ref:.4f}; alive {d[0]:.0f}/{d[3]:.0f} vs "
              f"{ref['d'][0]:.0f}/{ref['d'][3]:.0f}")
        assert abs(pk - pk_ref) <= tol_f * pk_ref
        assert abs(gain - g_ref) <= tol_g * abs(g_ref)
        assert abs(d[2] - s_ref) <= tol_g * s_ref
        assert abs(d[0] - ref["d"][0]) <= tol_n * cfg.n_beam and abs(d[3] - ref["d"][3]) <= tol_n * cfg.n_beam
    assert abs(g_ref) > 100.0 and s_ref > 10.0  # a measurable gain and spread after 1000 k_p^-1


def _batch_run(wk, cfgs, nsteps, sample):
    import torch
    keep = []
    for c in cfgs:
        nm = synth.plasma_normals(c)
        keep.append((None if nm is None else torch.from_numpy(nm).cuda(), torch.from_numpy(synth.beam_normals(c)).cuda()))
    torch.cuda.synchronize()
    with wk.Simulations(cfgs, wk.WAKE_MIXED) as s:
        for i, (tp, tb) in enumerate(keep):
            wk.wake_load_plasma(s.h, i, tp)
            wk.wake_load_beam(s.h, i, tb)
        d0 = s.diagnostics()
        wk.wake_step(s.h, nsteps)
        ms = wk.wake_step_kernel_ms(s.h)
        got = {i: (s.fields(i)["ez"].cpu().numpy(), s.diagnostics()[i]) for i in sample}
        for i in sample:
            assert s.status(i) == wk.WAKE_OK, wk.wake_last_error()
    return d0, got, ms


@pytest.mark.parametrize("pipelined", [True, False])
def test_batched_sweep_full_batch_sampled_simulations(wk, monkeypatch, pipelined):
    """Warm plasma over up to 4096 slices in FP32: the fields are held to 1% of peak |E_z|
    (the worst node error is ~1e-3 of peak on the longest boxes) and the witness energy gain
    to 0.5% of the FP64 oracle's."""
    if not pipelined:
        monkeypatch.setenv("WAKE_BATCH_PIPELINE", "0")
    cfgs = synth.config_batch()  # 256 simulations, as the benchmark
    nsteps = 2
    sample = [0, 101, 255]
    d0, got, ms = _batch_run(wk, cfgs, nsteps, sample)
    assert (ms > 0.0) == pipelined
    for i in sample:
        c = cfgs[i]
        pl = oracle.plasma_init(c, synth.plasma_normals(c))
        bm = oracle.beam_init(c, synth.beam_normals(c))
        ref = oracle.run(c, pl, bm, nsteps)
        dr = oracle.diagnostics(c, bm)
        ez, d = got[i]
        scale = np.abs(ref["ez"]).max()
        err = np.abs(ez - ref["ez"]).max() / scale
        print(f"sim {i} ({c.nr} x {c.nxi}, u_th {c.u_th:.4f}): max |dE_z| / peak = {err:.2e}")
        assert err <= 1e-2, i
        assert d[0] == dr[0] and d[3] == dr[3], i
        gain, gain_ref = d[1] - d0[i][1], dr[1] - d0[i][1]
        assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref) + 1e-9 * c.gamma_b, (i, gain, gain_ref)
