"""Pins of the oracle's slab geometry (x, xi) against what the mathematics fixes (no GPU).

Slab reading (Sec. I: WAKE handles slab as well as cylindrical geometry): d/dy = 0 in place of
d/dtheta = 0, x >= 0 with the mirror plane x = 0, hat volumes per unit area, lap_perp = d_x^2,
Eq. 6 as d_x B_y = d_xi^2 psi + J_z, the conserved u_y entering gamma only.  Each test pins one
part to something other than the oracle itself: the linear slab wake in closed form (Green's
function of d_x^2 - 1), its second-order convergence, the exact uniform density of the
unperturbed sheets, the QS invariant on test electrons pushed with the full equations of
motion in the oracle's fields, the Eq. 12 sheet bunch recovered by the beam deposit, and the
y = 0 plane kept by the Boris push.
"""
import math
import warnings

import numpy as np
import pytest

import oracle
import synth

warnings.filterwarnings("ignore", category=Warning, module="scipy")


def _slab_linear(nr, nxi, n0):
    import linear_theory as lt
    cfg = synth.config_slab_linear(nr=nr, nxi=nxi, n0=n0)
    out = oracle.march(cfg, oracle.plasma_init(cfg, None), oracle.nb_analytic(cfg))
    return cfg, out, lt.slab_linear_fields(cfg)


def _rel_err(cfg, out, ref, key, xfrac=0.7, imin=0):
    ic = int(xfrac * cfg.nr)
    d = np.abs(out[key] - ref[key])[:, imin:ic]
    return d.max() / np.abs(ref[key]).max()


def test_slab_linear_wake_matches_closed_form():
    """A weak sheet driver (n_b/n_p = 1e-6): psi, E_z, B_y and E_x match the conducting-wall
    slab linear theory to the discretisation error."""
    cfg, out, ref = _slab_linear(128, 256, 1e-6)
    errs = {k: _rel_err(cfg, out, ref, k) for k in ("psi", "ez", "bth", "er")}
    assert errs["psi"] < 5e-3 and errs["ez"] < 5e-3, errs
    assert errs["bth"] < 5e-3 and errs["er"] < 1.5e-2, errs
    # the cylindrical operators give a different wake: the slab branch is the one that ran
    cyl = oracle.march(synth.config_linear(nr=128, nxi=256, n0=1e-6),
                       oracle.plasma_init(synth.config_linear(nr=128, nxi=256, n0=1e-6), None),
                       oracle.nb_analytic(synth.config_linear(nr=128, nxi=256, n0=1e-6)))
    assert np.abs(cyl["psi"] - ref["psi"]).max() > 20 * np.abs(out["psi"] - ref["psi"]).max()


def test_slab_linear_wake_second_order_convergence():
    """Halving (dx, dxi) cuts the closed-form error by about 4 for every field."""
    errs = {k: [] for k in ("psi", "ez", "bth", "er")}
    for nr in (32, 64, 128):
        cfg, out, ref = _slab_linear(nr, 2 * nr, 1e-6)
        for k in errs:
            errs[k].append(_rel_err(cfg, out, ref, k))
    for k, e in errs.items():
        assert math.log2(e[1] / e[2]) > 1.6, (k, e)


def test_slab_unperturbed_sheets_have_unit_density():
    """Cold sheets at the cell midpoints, hat-deposited and divided by the slab hat widths
    (dx, halved on the mirror plane and at the wall), give n = 1 at every node exactly; their
    weights add up to the ion charge per unit area, L."""
    cfg = synth.config_slab_linear(nr=40, nxi=8)
    pl = oracle.plasma_init(cfg, None)
    assert abs(pl["w"].sum() - cfg.rmax) < 1e-12
    assert np.all(pl["l"] == 0.0)
    rho = oracle.deposit_charge(cfg, pl["r0"], pl["w"])
    dx = cfg.rmax / cfg.nr
    vol = np.full(cfg.nr + 1, dx)
    vol[0] = vol[-1] = 0.5 * dx
    assert np.abs(rho / vol - 1.0).max() < 1e-13
    # warm sheets: the weight of each is dx / ppc times the flux factor Gamma0 / gamma0
    cfgw = synth.config_slab_linear(nr=40, nxi=8)
    cfgw.u_th, cfgw.ppc = 0.05, 4
    nm = np.random.default_rng(3).standard_normal((cfgw.nr * cfgw.ppc, 3))
    pw = oracle.plasma_init(cfgw, nm)
    u = 0.05 * nm
    g0 = np.sqrt(1 + (u * u).sum(1))
    assert np.allclose(pw["w"], dx / cfgw.ppc * (g0 - u[:, 2]) / g0, rtol=1e-14)
    assert np.allclose(pw["l"], u[:, 1], rtol=0, atol=0)  # l holds the conserved u_y


def _slab_invariant_drift(cfg, out, scale_ez=1.0):
    from scipy.interpolate import RegularGridInterpolator as RGI
    x = np.arange(cfg.nr + 1) * cfg.rmax / cfg.nr
    xi = np.arange(cfg.nxi + 1) * cfg.ximax / cfg.nxi
    F = {k: RGI((xi, x), out[k] * (scale_ez if k == "ez" else 1.0)) for k in ("er", "ez", "bth", "psi")}
    x0 = np.array([0.05, 0.3, 0.5, 0.8, 1.2])
    y = np.stack([x0, 0 * x0, 0 * x0, 1 + 0 * x0], 1)

    def rhs(s, y):  # full equations of motion of a plasma electron in (x, xi), d/dxi
        ax = np.abs(y[:, 0])
        sg = np.where(y[:, 0] < 0, -1.0, 1.0)  # E_x and B_y are odd in x
        pts = np.stack([np.full(len(y), s), ax], 1)
        Ex, Ez, By = sg * F["er"](pts), F["ez"](pts), sg * F["bth"](pts)
        ux, uz, g = y[:, 1], y[:, 2], y[:, 3]
        G = g - uz
        return np.stack([ux / G, -(g * Ex - uz * By) / G, -(g * Ez + ux * By) / G, -(ux * Ex + uz * Ez) / G], 1)

    h = cfg.ximax / cfg.nxi
    worst = 0.0
    for k in range(cfg.nxi):
        s = k * h
        k1 = rhs(s, y)
        k2 = rhs(s + h / 2, y + h / 2 * k1)
        k3 = rhs(s + h / 2, y + h / 2 * k2)
        k4 = rhs(s + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        psi = F["psi"](np.stack([np.full(len(y), s + h), np.abs(y[:, 0])], 1))
        worst = max(worst, np.abs(y[:, 3] - y[:, 2] - psi - 1.0).max())
    return worst


def test_slab_qs_invariant_on_test_electrons():
    """Eq. 1 in the slab: electrons pushed with the full equations of motion (du_z/dxi and
    dgamma/dxi from the Lorentz force of E_x, E_z, B_y) through the oracle's slab fields keep
    gamma - u_z - psi = 1 to O(dxi^2), across the mirror plane; a 2% error in E_z breaks it."""
    drifts = []
    for nr in (64, 128):
        cfg = synth.config_slab_linear(nr=nr, nxi=2 * nr, n0=0.5)
        out = oracle.march(cfg, oracle.plasma_init(cfg, None), oracle.nb_analytic(cfg))
        drifts.append(_slab_invariant_drift(cfg, out))
    assert drifts[1] < 6e-4 and drifts[1] < drifts[0] / 2, drifts
    assert _slab_invariant_drift(cfg, out, scale_ez=1.02) > 10 * drifts[1]


def test_slab_sheet_beam_density_and_weights():
    """The Gaussian sheet bunch folded onto x >= 0 and deposited with the slab hat widths
    recovers Eq. 12: n_d on the mirror plane at the bunch centre, and the exp(-x^2/2 sigma^2)
    profile; the weight carries the half-slab integral sigma sqrt(2 pi)/2 (a factor 2 off
    in it, or a full hat width on x = 0, fails)."""
    cfg = synth.config_slab_linear(nr=32, nxi=64, n0=0.7)
    cfg.n_beam = cfg.n_drive = 400_000
    cfg.eps_n = 0.0
    nm = np.random.default_rng(5).standard_normal((5, cfg.n_beam))
    b = oracle.beam_init(cfg, nm)
    assert np.all(b["y"] == 0.0) and np.all(b["uy"] == 0.0)
    wd, _ = oracle.beam_weights(cfg)
    assert abs(wd - cfg.n_d * math.pi * cfg.sigma_r * cfg.sigma_zd / cfg.n_beam) < 1e-15
    nb = oracle.beam_deposit(cfg, b)
    ref = oracle.nb_analytic(cfg)
    k = int(round(cfg.xi_d / (cfg.ximax / cfg.nxi)))
    band = slice(k - 2, k + 3)
    # hat deposit smooths by a cell; sampling noise ~ 1/sqrt(particles per node)
    assert np.abs(nb[band, :8] - ref[band, :8]).max() < 0.04 * cfg.n_d
    assert abs(nb[k, 0] / ref[k, 0] - 1.0) < 0.04


def test_slab_boris_push_stays_in_the_xz_plane():
    """The slab fields have no y component (E = (E_x, 0, E_z), B = (0, B_y, 0)): a sheet-beam
    particle keeps y = u_y = 0 exactly, and its x-z motion is the cylindrical push at y = 0."""
    cfg = synth.config_slab_linear(nr=16, nxi=16)
    cfg.n_beam = cfg.n_drive = 64
    rng = np.random.default_rng(9)
    nm = rng.standard_normal((5, cfg.n_beam))
    b = oracle.beam_init(cfg, nm)
    shape = (cfg.nxi + 1, cfg.nr + 1)
    f = {k: rng.uniform(-0.3, 0.3, shape) for k in ("er", "ez", "bth")}
    c = {k: v.copy() for k, v in b.items()}
    for _ in range(5):
        oracle.beam_push(cfg, b, f)
    assert np.all(b["y"] == 0.0) and np.all(b["uy"] == 0.0)
    cyl = synth.config_linear(nr=16, nxi=16)
    cyl.n_beam = cyl.n_drive = 64
    cyl.ds = cfg.ds
    for _ in range(5):
        oracle.beam_push(cyl, c, f)
    for k in ("x", "ux", "uz", "xi"):
        assert np.array_equal(b[k], c[k]), k


def test_slab_refuses_trapping():
    """Trapping is read for the cylinder only: the slab march with a threshold is refused."""
    cfg = synth.config_slab_linear(nr=16, nxi=16)
    with pytest.raises(oracle.OracleError):
        oracle.march_trap(cfg, oracle.plasma_init(cfg, None), oracle.nb_analytic(cfg), 1.5, 10)


def test_slab_warm_neutral_plasma_stays_quiet():
    """With no driver, warm sheets (u_th = 0.05, mirrored momentum pairs) keep the fields at
    the thermal noise level, |psi|, |E_z|, |B_y| < 0.25 u_th over 128 slices: u_y enters gamma
    only, with no centrifugal push and no displacement (either would sweep the sheets off the
    mirror plane and raise psi to order one)."""
    cfg = synth.config_slab_linear(nr=64, nxi=128, n0=0.0)
    cfg.u_th, cfg.ppc = 0.05, 8
    out = oracle.march(cfg, oracle.plasma_init(cfg, synth.plasma_normals(cfg)), np.zeros((cfg.nxi + 1, cfg.nr + 1)))
    for k in ("psi", "ez", "bth"):
        assert np.abs(out[k]).max() < 0.25 * cfg.u_th, (k, np.abs(out[k]).max())


def test_slab_uniform_y_drift_is_an_equilibrium():
    """Cold sheets all drifting with the same u_y = 1 (gamma_0 = Gamma_0 = sqrt 2, u_z = 0) and
    no driver: by d/dy = 0 nothing depends on y, so there is no force, no current but the
    uniform J_y that no field here sees, and every field stays exactly zero.  A u_y that moved
    a sheet (a cylindrical frame), or a stage that lost it from gamma (J_z != 0), would not."""
    cfg = synth.config_slab_linear(nr=32, nxi=64, n0=0.0)
    pl = oracle.plasma_init(cfg, None)
    U = 1.0
    pl["l"][:] = U
    pl["G0"][:] = math.sqrt(1.0 + U * U)
    out = oracle.march(cfg, pl, np.zeros((cfg.nxi + 1, cfg.nr + 1)), traj=True)
    for k in ("psi", "ez", "bth", "er"):
        assert np.abs(out[k]).max() < 1e-14, (k, np.abs(out[k]).max())
    assert np.array_equal(out["traj"][-1, 0], pl["r0"])
