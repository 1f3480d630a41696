"""The ring trajectory dump (Sec. IV, Figs. 4-5) through the C ABI: against the oracle's
trajectories on the same seeded plasma, and the axis crossing the paper reads off them.

FP64 form: every dumped r, u_r and Gamma agrees with the oracle to 1e-8 of its scale.  Mixed
form: in the linear case to a small fraction of a cell; in blowout the rings that recross the
axis do so chaotically, so the mixed form is held to the crossing statistics (where each ring
crosses, the length of the axis-crossing region) and to most rings staying close.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1411_3246_gb300 import studies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _oracle_traj(cfg, nm):
    return oracle.march(cfg, oracle.plasma_init(cfg, nm), oracle.nb_analytic(cfg), traj=True)["traj"]


@pytest.mark.parametrize("every", [1, 3])
def test_traj_fp64_matches_oracle(wk, every):
    cfg = synth.config_blowout(n_beam=0, nr=64, nxi=128)  # warm, two-bunch frozen driver
    nm = synth.plasma_normals(cfg)
    ref = _oracle_traj(cfg, nm)[::every]
    xi, tr = studies.trajectories(cfg, nm, every, wk.WAKE_FP64)
    assert tr.shape == ref.shape and xi[1] == every * cfg.ximax / cfg.nxi
    for q in range(3):
        scale = np.abs(ref[:, q]).max()
        assert np.abs(tr[:, q] - ref[:, q]).max() <= 1e-8 * scale, q


def test_traj_mixed_linear_within_small_fraction_of_cell(wk):
    cfg = synth.config_linear()
    ref = _oracle_traj(cfg, None)
    _, tr = studies.trajectories(cfg, None, 1, wk.WAKE_MIXED)
    dr = cfg.rmax / cfg.nr
    assert np.abs(tr[:, 0] - ref[:, 0]).max() <= 1e-4 * dr
    assert np.abs(tr[:, 1] - ref[:, 1]).max() <= 1e-4 * np.abs(ref[:, 1]).max()
    assert np.abs(tr[:, 2] - ref[:, 2]).max() <= 1e-5 * np.abs(ref[:, 2]).max()


def test_traj_mixed_blowout_crossing_statistics(wk):
    """Warm blowout (the Table I driver frozen in a 5 eV plasma, 128 x 512): the mixed form's
    rings cross the axis behind the drive bunch at the oracle's slice (within one slice) for
    90% of the crossing rings; the crossing region has the oracle's length within one slice and
    the same crossing charge within 5%; 90% of the rings stay within 0.5% of a cell of the
    oracle's radius over the whole box (the rest recross the axis chaotically)."""
    cfg = synth.config_table1(nr=128, nxi=512, u_th=float(np.sqrt(5.0 / 511.0e3)))
    nm = synth.plasma_normals(cfg)
    ref = _oracle_traj(cfg, nm)
    xi, tr = studies.trajectories(cfg, nm, 1, wk.WAKE_MIXED)
    w = ref[0, 0]  # ring charge is proportional to its initial radius (flux factor ~1)
    after = cfg.xi_d + cfg.sigma_zd
    xr = studies.axis_crossings(ref[:, 0], xi, after, 0.1)
    xg = studies.axis_crossings(tr[:, 0], xi, after, 0.1)
    wr, fr = studies.crossing_width(xr, w)
    wg, fg = studies.crossing_width(xg, w)
    dxi = cfg.ximax / cfg.nxi
    assert np.isfinite(xr).sum() >= 8 and fr > 0
    both = np.isfinite(xr) & np.isfinite(xg)
    assert np.mean(np.abs(xr[both] - xg[both]) <= 1.01 * dxi) >= 0.9
    assert abs(fg - fr) <= 0.05 * fr
    assert abs(wg - wr) <= 1.01 * dxi, (wg, wr)
    dr = cfg.rmax / cfg.nr
    dev = np.abs(tr[:, 0] - ref[:, 0]).max(axis=0)
    assert np.quantile(dev, 0.9) <= 5e-3 * dr


def test_invalid_traj_calls(wk):
    import torch
    cfg = synth.config_linear(nr=32, nxi=16)
    with wk.Simulations([cfg], wk.WAKE_MIXED) as s:
        out = torch.empty((17, 3, cfg.nr * cfg.ppc), dtype=torch.float64, device="cuda")
        with pytest.raises(wk.WakeError) as e:
            wk.wake_plasma_march_traj(s.h, 0, 1, out)  # no plasma yet
        assert e.value.code == wk.WAKE_ESTATE
        wk.wake_load_plasma(s.h, 0, None)
        with pytest.raises(wk.WakeError) as e:
            wk.wake_plasma_march_traj(s.h, 0, 0, out)
        assert e.value.code == wk.WAKE_EINVAL
        with pytest.raises(wk.WakeError) as e:
            wk.wake_plasma_march_traj(s.h, 1, 1, out)
        assert e.value.code == wk.WAKE_EINVAL
    big = synth.config_large(n_beam=0)  # 2049 nodes: the wide form, no one-CTA tile
    with wk.Simulations([big], wk.WAKE_MIXED) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(synth.plasma_normals(big)).cuda())
        with pytest.raises(wk.WakeError) as e:
            wk.wake_plasma_march_traj(s.h, 0, 64, out)
        assert e.value.code == wk.WAKE_EINVAL


def test_axis_crossing_broadens_with_temperature(wk):
    """Sec. IV (Figs. 4 and 5), Table I driver frozen: the plasma electrons expelled by the
    drive bunch fall back and cross the axis behind it; at 5 eV they cross over a broader
    region than in a cold plasma, and with a single bunch (n_w = 0) the cold crossing is
    narrower than with two."""
    widths = {}
    for bunches in ("two", "one"):
        for te in (0.0, 5.0):
            cfg = synth.config_table1(nr=256, nxi=1024, u_th=float(np.sqrt(te / 511.0e3)))
            if bunches == "one":
                cfg.n_w = 0.0
            nm = synth.plasma_normals(cfg) if te > 0 else None
            xi, tr = studies.trajectories(cfg, nm, 1, wk.WAKE_MIXED)
            xc = studies.axis_crossings(tr[:, 0], xi, cfg.xi_d + cfg.sigma_zd, 0.1)
            widths[bunches, te] = studies.crossing_width(xc, tr[0, 0])
    print("axis-crossing widths (k_p^-1, charge fraction):", widths)
    assert widths["two", 5.0][0] > 1.3 * widths["two", 0.0][0]
    assert widths["one", 5.0][0] > 1.3 * widths["one", 0.0][0]
    assert widths["one", 0.0][0] < widths["two", 0.0][0]
