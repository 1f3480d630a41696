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


def test_axis_crossings_of_constructed_trajectories():
    """Rings whose radii dip to a known minimum at known slices: the first minimum behind
    xi_after and below r_cut is found; a ring that stays away from the axis has none; a dip
    ahead of xi_after does not count."""
    xi = np.linspace(0.0, 10.0, 101)
    r = np.empty((101, 4))
    r[:, 0] = np.abs(xi - 6.0) + 0.0          # V-shaped crossing at xi = 6
    r[:, 1] = np.abs(xi - 6.5) * 0.5 + 0.01   # crossing at 6.5, minimum radius 0.01
    r[:, 2] = 2.0 + 0.1 * np.sin(xi)          # never near the axis
    r[:, 3] = np.minimum(np.abs(xi - 1.0), np.abs(xi - 7.0))  # dips at 1 (ahead) and at 7
    xc = studies.axis_crossings(r, xi, xi_after=3.0, r_cut=0.05)
    assert xc[0] == xi[60] and xc[1] == xi[65] and np.isnan(xc[2]) and xc[3] == xi[70]


def test_crossing_width_weighted_quantiles():
    """Charge-weighted 10-90% range: uniform crossings over [2, 4] with equal weights give a
    width of 1.6; giving all weight to one point gives 0; uncrossed rings are left out."""
    x = np.linspace(2.0, 4.0, 2001)
    w = np.ones_like(x)
    width, frac = studies.crossing_width(x, w)
    assert abs(width - 1.6) < 2e-3 and frac == 1.0
    x2 = np.concatenate([x, [np.nan] * 2001])
    width2, frac2 = studies.crossing_width(x2, np.ones_like(x2))
    assert abs(width2 - 1.6) < 2e-3 and abs(frac2 - 0.5) < 1e-12
    w3 = np.zeros_like(x)
    w3[1000] = 1.0
    assert studies.crossing_width(x, w3)[0] == 0.0
