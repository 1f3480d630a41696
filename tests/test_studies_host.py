"""Host-side reductions of the parameter studies (no GPU): distances to beam steps, the spike
and flat-region reading of an on-axis E_z profile, witness energies and the spectrum peak,
each on an input whose answer is known by construction."""
import math

import numpy as np

import synth
from paper_1411_3246_gb300 import studies


def test_units_follow_the_table1_plasma():
    # Sec. III: k_p^-1 = 23.7 um at n_p = 5e16 cm^-3; E_0 = 96 sqrt(n_p) V/m = 21.47 GV/m
    assert studies.KP_INV_M == 23.7e-6
    assert abs(studies.E0_GV_PER_M - 21.4663) < 1e-3
    # 1.14 m at ds = 5 k_p^-1: 1.14 / 23.7e-6 / 5 = 9620.3 steps
    assert studies.steps_for_length(1.14, 5.0) == 9620
    assert studies.steps_for_length(1.49, 5.0) == 12574


def test_spike_and_flat_of_a_constructed_profile():
    cfg = synth.config_table1(nr=16, nxi=1024)
    xi = np.arange(cfg.nxi + 1) * cfg.ximax / cfg.nxi
    ez = np.zeros_like(xi)
    core = np.abs(xi - cfg.xi_w) < 0.25 * cfg.sigma_zw
    ez[core] = -0.7
    ez[np.argmin(np.abs(xi - (cfg.xi_w - 1.0)))] = -1.6  # a one-node spike ahead of the witness
    ez[np.argmin(np.abs(xi - 2.0))] = 0.4                # decelerating field in the driver
    spike, flat = studies.spike_and_flat(ez, cfg)
    assert spike == 1.6 and abs(flat - 0.7) < 1e-15


def test_witness_energies_and_spectrum_peak():
    rng = np.random.default_rng(7)
    n_drive, n_w = 1000, 20000
    gam = np.concatenate([np.full(n_drive, 1.0e4), rng.normal(40.6 / studies.MC2_GEV, 300.0, n_w)])
    uz = np.sqrt(gam * gam - 1.0)  # u_perp = 0: gamma = sqrt(1 + u_z^2)
    xyz = np.zeros((6, n_drive + n_w))
    xyz[5] = uz
    lost = np.zeros(n_drive + n_w, dtype=np.uint8)
    lost[n_drive:n_drive + 500] = 1  # lost witness particles are left out
    e = studies.witness_energies_gev(xyz, lost, n_drive)
    assert e.size == n_w - 500
    np.testing.assert_allclose(e, studies.MC2_GEV * gam[n_drive + 500:], rtol=1e-14)
    # a narrow line at 40.6 GeV (sigma 0.15 GeV) on a flat background: the fullest 0.25 GeV bin
    e = np.concatenate([e, rng.uniform(20.0, 60.0, 20000)])
    assert abs(studies.spectrum_peak(e) - 40.6) <= 0.25
    # and the bin centres are on the 0.25 GeV grid
    assert abs(studies.spectrum_peak(np.array([44.6, 44.6, 10.0])) - 44.625) < 1e-12


def test_facet_config_splits_particles_by_charge():
    cfg = synth.config_facet(n_beam=1 << 20, te_ev=5.0)
    q_ratio = (2.85 * 0.81) / (3.56 * 1.44)  # Table I: n_w sigma_zw / (n_d sigma_zd)
    n_w = cfg.n_beam - cfg.n_drive
    assert abs(n_w / cfg.n_drive - q_ratio) < 1e-5
    assert cfg.eps_n == 0.0 and abs(cfg.u_th - math.sqrt(5.0 / 511.0e3)) < 1e-15
    assert abs(cfg.gamma_b * 0.511e-3 - 23.0) < 1e-9
