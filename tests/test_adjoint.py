"""The adjoint's arithmetic (paper_1411_3246_gb300/csrc/adjoint_core.h, host build) against
central finite differences of the FP64 oracle: gradients of the witness mean energy gain and
rms energy spread after a few beam steps with respect to n_w, the witness delay, sigma_zd,
u_th and a 4-bin witness current profile.

Step size: h = 1e-4 relative.  At h = 1e-6 the differences of the rms spread are dominated
by rounding (a sweep over h = 1e-4 .. 1e-7 shows the adjoint value at 1e-4 and 1e-5 and
drifts below), and the truncation error at 1e-4 is below 1e-7 relative.
"""
import numpy as np
import pytest

import adjoint_host
import oracle
import synth


def adjoint_case(nr=16, nxi=32, n_beam=512):
    cfg = synth.config_batch(n_sims=1)[0]
    cfg.nr, cfg.nxi = nr, nxi
    cfg = synth.two_bunch(cfg, 0.3, cfg.xi_w - cfg.xi_d, n_beam)
    cfg.u_th = 0.005  # away from 0, where the Maxwellian's dependence is not smooth in sign
    return cfg


def theta_of(cfg):
    return np.array([cfg.n_w, cfg.xi_w - cfg.xi_d, cfg.sigma_zd, cfg.u_th])


def oracle_fd(cfg, nsteps, theta, profile, nm_p, nm_b, dobs, rel=1e-4):
    x = np.concatenate([theta, profile])
    g = np.zeros_like(x)
    for i in range(len(x)):
        h = rel * max(abs(x[i]), 1e-3)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        op = oracle.witness_objective(cfg, xp[:4], xp[4:], nm_p, nm_b, nsteps)
        om = oracle.witness_objective(cfg, xm[:4], xm[4:], nm_p, nm_b, nsteps)
        g[i] = np.dot(dobs, (op - om) / (2 * h))
    return g


def assert_grad_close(g, ref, rtol=1e-4):
    floor = 1e-3 * np.abs(ref).max()  # components far below the largest one: absolute check
    bad = np.abs(g - ref) > rtol * np.maximum(np.abs(ref), floor)
    assert not bad.any(), (np.nonzero(bad)[0], g, ref)


def test_host_adjoint_forward_equals_oracle_objective():
    cfg = adjoint_case()
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    prof = np.array([1.0, 0.8, 1.3, 1.1])
    obs, _ = adjoint_host.gradient(cfg, 3, theta_of(cfg), prof, nm_p, nm_b)
    ref = oracle.witness_objective(cfg, theta_of(cfg), prof, nm_p, nm_b, 3)
    np.testing.assert_allclose(obs, ref, rtol=1e-9)


@pytest.mark.parametrize("dobs", [(1.0, 0.0), (0.0, 1.0), (0.5, -2.0)])
def test_host_adjoint_matches_oracle_finite_differences(dobs):
    cfg = adjoint_case()
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    theta, prof = theta_of(cfg), np.ones(4)
    _, g = adjoint_host.gradient(cfg, 3, theta, prof, nm_p, nm_b, np.array(dobs))
    ref = oracle_fd(cfg, 3, theta, prof, nm_p, nm_b, np.array(dobs))
    assert_grad_close(g, ref)


def test_host_adjoint_gradient_is_linear_in_the_seed():
    cfg = adjoint_case()
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    theta, prof = theta_of(cfg), np.ones(4)
    g = [adjoint_host.gradient(cfg, 2, theta, prof, nm_p, nm_b, np.array(d))[1] for d in ((1, 0), (0, 1), (3, -1))]
    np.testing.assert_allclose(g[2], 3 * g[0] - g[1], rtol=1e-9, atol=1e-12 * np.abs(g[0]).max())
