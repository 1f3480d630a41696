"""The adjoint form through the C ABI (wake_adjoint_*) and its torch.autograd binding: the
CUDA gradient equals the host build of the same arithmetic and central finite differences
of the FP64 oracle."""
import numpy as np
import pytest

import adjoint_host
import oracle
import synth
from test_adjoint import adjoint_case, assert_grad_close, oracle_fd, theta_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _adj(wk, cfg, nsteps, nbins):
    import torch
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).cuda()
    return wk.Adjoint(cfg, nsteps, nbins, nm_p, nm_b)


def test_gpu_adjoint_equals_host_build(wk):
    cfg = adjoint_case(nr=32, nxi=96, n_beam=4096)
    theta = theta_of(cfg)
    prof = np.linspace(0.7, 1.3, 8)
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    for dobs in ((1.0, 0.0), (0.0, 1.0)):
        o_h, g_h = adjoint_host.gradient(cfg, 4, theta, prof, nm_p, nm_b, np.array(dobs))
        with _adj(wk, cfg, 4, 8) as a:
            o = np.array(a.forward(theta, prof))
            g = np.array(a.backward(dobs))
        np.testing.assert_allclose(o, o_h, rtol=1e-10)
        assert np.abs(g - g_h).max() <= 1e-8 * np.abs(g_h).max(), (g, g_h)


def test_gpu_adjoint_matches_oracle_finite_differences(wk):
    cfg = adjoint_case()
    theta, prof = theta_of(cfg), np.ones(4)
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    dobs = np.array([1.0, -0.5])
    with _adj(wk, cfg, 3, 4) as a:
        obs = np.array(a.forward(theta, prof))
        g = np.array(a.backward(dobs))
    np.testing.assert_allclose(obs, oracle.witness_objective(cfg, theta, prof, nm_p, nm_b, 3), rtol=1e-9)
    assert_grad_close(g, oracle_fd(cfg, 3, theta, prof, nm_p, nm_b, dobs))


def test_autograd_function_gives_the_adjoint_gradient(wk):
    """The autograd binding returns the adjoint's gradient, which central differences of the
    library's own forward confirm (a case with few beam particles, so that the h-shift moves
    no particle across a cell edge, where the linear hats have a kink)."""
    import torch
    cfg = adjoint_case(nr=16, nxi=40, n_beam=512)
    with _adj(wk, cfg, 3, 6) as a:
        th = torch.tensor(theta_of(cfg), dtype=torch.float64, device="cuda", requires_grad=True)
        pr = torch.ones(6, dtype=torch.float64, device="cuda", requires_grad=True)
        obs = wk.witness_observables(a, th, pr)
        loss = obs[0] - 0.5 * obs[1]
        loss.backward()
        g = a.backward([1.0, -0.5])
        # finite differences of the library's own forward
        x0 = np.concatenate([theta_of(cfg), np.ones(6)])
        fd = np.zeros_like(x0)
        for i in range(len(x0)):
            h = 1e-4 * max(abs(x0[i]), 1e-3)
            xp, xm = x0.copy(), x0.copy()
            xp[i] += h
            xm[i] -= h
            op, om = np.array(a.forward(xp[:4], xp[4:])), np.array(a.forward(xm[:4], xm[4:]))
            fd[i] = ((op[0] - 0.5 * op[1]) - (om[0] - 0.5 * om[1])) / (2 * h)
    got = np.concatenate([th.grad.cpu().numpy(), pr.grad.cpu().numpy()])
    np.testing.assert_allclose(got, g, rtol=1e-12)
    assert_grad_close(got, fd)


def test_adjoint_bench_size_against_oracle(wk):
    """The differentiation workload the benchmark times (128 x 1024, 262,144 beam particles,
    100 steps, 64 profile bins): the forward observables against the oracle's to 1e-9, and
    gradient components against central differences of the oracle (h = 1e-4 relative; the
    oracle runs in worker processes).  The mean-gain components to 5e-3 (their differences at
    h = 1e-3 and 1e-4 agree to 1e-3 at worst, a profile bin's).  The spread is
    piecewise smooth only (the linear hats' kinks under a quarter million particles):
    differences at h = 1e-3, 1e-4 and 1e-5 of its n_w component spread by 1.3%, so its
    components are held to 3e-2.  The u_th components are not compared here: there every ring
    moves, and the difference quotients at those three h disagree by a factor of six."""
    import oracle_jobs
    cfg = synth.config_adjoint()
    nsteps, nbins = cfg.n_steps, 64
    theta, prof = theta_of(cfg), np.ones(nbins)
    x0 = np.concatenate([theta, prof])
    comps = [0, 1, 4 + 20, 4 + 32]  # n_w, delay and two profile bins
    jobs = [(x0[:4], x0[4:])]
    steps = []
    for i in comps:
        h = 1e-4 * max(abs(x0[i]), 1e-3)
        steps.append(h)
        for sgn in (1.0, -1.0):
            x = x0.copy()
            x[i] += sgn * h
            jobs.append((x[:4], x[4:]))
    with oracle_jobs.pool(len(jobs)) as pool:
        res = [pool.apply_async(oracle_jobs.witness_objective, (cfg, th, pr, nsteps)) for th, pr in jobs]
        with _adj(wk, cfg, nsteps, nbins) as a:
            obs = np.array(a.forward(theta, prof))
            g_mean = np.array(a.backward([1.0, 0.0]))
            g_spread = np.array(a.backward([0.0, 1.0]))
        vals = [np.array(r.get(timeout=1800)) for r in res]
    np.testing.assert_allclose(obs, vals[0], rtol=1e-9)
    for n, (i, h) in enumerate(zip(comps, steps)):
        fd = (vals[1 + 2 * n] - vals[2 + 2 * n]) / (2 * h)
        print(f"component {i}: adjoint {g_mean[i]:.6g}, {g_spread[i]:.6g}; oracle differences {fd[0]:.6g}, {fd[1]:.6g}")
        assert abs(g_mean[i] - fd[0]) <= 5e-3 * abs(fd[0]), (i, g_mean[i], fd[0])
        assert abs(g_spread[i] - fd[1]) <= 3e-2 * abs(fd[1]), (i, g_spread[i], fd[1])


@pytest.mark.parametrize("full_tape", ["1", "0"])
def test_pipelined_adjoint_equals_sequential(wk, monkeypatch, full_tape):
    """The pipelined adjoint (one CTA per beam step, many steps at once; the default), with
    every slice kept on the tape (the default when it fits) or with checkpoints every
    ~sqrt(Nxi) slices recomputed in the reverse (WAKE_ADJOINT_FULL_TAPE=0), against the same
    handle run one step at a time (WAKE_ADJOINT_PIPELINE=0); both variables are read by
    wake_adjoint_init.  The observables and the gradient agree to rounding (only the order of
    the atomic sums differs)."""
    cfg = adjoint_case(nr=32, nxi=128, n_beam=8192)
    theta, prof = theta_of(cfg), np.linspace(0.8, 1.2, 8)
    out = []
    monkeypatch.setenv("WAKE_ADJOINT_FULL_TAPE", full_tape)
    for pipe in ("1", "0"):
        monkeypatch.setenv("WAKE_ADJOINT_PIPELINE", pipe)
        with _adj(wk, cfg, 12, 8) as a:
            o = np.array(a.forward(theta, prof))
            g = np.array(a.backward([1.0, -0.5]))
        out.append((o, g))
    (o1, g1), (o0, g0) = out
    np.testing.assert_allclose(o1, o0, rtol=1e-11)
    assert np.abs(g1 - g0).max() <= 1e-9 * np.abs(g0).max(), (g1, g0)


def test_adjoint_pipeline_wait_runs_out(wk, monkeypatch):
    """WAKE_SPIN_LIMIT=0 makes each wait of the pipelined adjoint poll once: the forward
    reports WAKE_ETIMEOUT and leaves cleanly; a fresh handle with the default limit runs."""
    cfg = adjoint_case(nr=32, nxi=256, n_beam=4096)
    theta, prof = theta_of(cfg), np.ones(4)
    monkeypatch.setenv("WAKE_SPIN_LIMIT", "0")
    with _adj(wk, cfg, 8, 4) as a:
        with pytest.raises(wk.WakeError) as e:
            a.forward(theta, prof)
        assert e.value.code == wk.WAKE_ETIMEOUT
    monkeypatch.delenv("WAKE_SPIN_LIMIT")
    with _adj(wk, cfg, 8, 4) as a:
        obs = np.array(a.forward(theta, prof))
        assert np.isfinite(obs).all()
        assert np.isfinite(np.array(a.backward([1.0, 0.0]))).all()
