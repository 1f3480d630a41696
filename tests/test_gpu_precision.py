"""The two precision splits of the FP32 form against the FP64 oracle, through the C ABI.

WAKE_MIXED keeps the radial solves on the FP32 pipe (charge sums in exact fixed point, scans
in float-float, the tridiagonal solve by FP32 cyclic reduction on row sums); WAKE_MIXED64 is
the split in which only the particle arithmetic is FP32 (sums across rings, scans and the
tridiagonal solve in FP64).  Both are held to the same per-result tolerances: fields within
1e-5 of peak |E_z| in the linear case; in blowout, peak E_z within 1% and the witness mean
energy gain and spread within 0.5%.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FORMS = ["mixed", "mixed64"]


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _prec(wk, form):
    return wk.WAKE_MIXED if form == "mixed" else wk.WAKE_MIXED64


def _march(wk, cfg, prec, nm):
    import torch
    with wk.Simulations([cfg], prec) as s:
        wk.wake_load_plasma(s.h, 0, None if nm is None else torch.from_numpy(nm).cuda())
        wk.wake_plasma_march(s.h)
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    return f


@pytest.mark.parametrize("form", FORMS)
def test_linear_fields_within_1e5_of_peak(wk, form):
    cfg = synth.config_linear()
    ref = oracle.march(cfg, oracle.plasma_init(cfg, None), oracle.nb_analytic(cfg))
    f = _march(wk, cfg, _prec(wk, form), None)
    scale = np.abs(ref["ez"]).max()
    errs = {k: np.abs(f[k] - ref[k]).max() / scale for k in ("psi", "ez", "er", "bth")}
    print(form, "linear, max node error / peak |E_z|:", errs)
    assert max(errs.values()) <= 1e-5, errs


@pytest.mark.parametrize("form", FORMS)
def test_blowout_march_full_size_peak_ez(wk, form):
    cfg = synth.config_blowout(n_beam=0)
    nm = synth.plasma_normals(cfg)
    ref = oracle.march(cfg, oracle.plasma_init(cfg, nm), oracle.nb_analytic(cfg))
    f = _march(wk, cfg, _prec(wk, form), nm)
    peak_ref = np.abs(ref["ez"][:, 0]).max()
    peak = np.abs(f["ez"][:, 0]).max()
    node = np.abs(f["ez"] - ref["ez"]).max() / peak_ref
    print(form, f"blowout 512 x 2048: peak E_z {peak:.6f} vs {peak_ref:.6f}, max node error / peak {node:.2e}")
    assert abs(peak - peak_ref) <= 0.01 * peak_ref
    k = int(round(cfg.xi_w / cfg.ximax * cfg.nxi))
    assert abs(f["ez"][k, 0] - ref["ez"][k, 0]) <= 0.01 * peak_ref


@pytest.mark.parametrize("form", FORMS)
def test_beam_steps_witness_energy(wk, form):
    """Pipelined steps over a box of 128 x 512 with 2^16 beam particles and ds = 50: the
    witness mean energy gain and rms spread within 0.5% of the oracle's."""
    import torch
    cfg = synth.config_blowout(n_beam=1 << 16, nr=128, nxi=512)
    cfg.ds = 50.0
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    pl, bm = oracle.plasma_init(cfg, nm_p), oracle.beam_init(cfg, nm_b)
    d0 = oracle.diagnostics(cfg, bm)
    oracle.run(cfg, pl, bm, 4)
    d_ref = oracle.diagnostics(cfg, bm)
    with wk.Simulations([cfg], _prec(wk, form)) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, 4)
        diag = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    gain_ref, gain = d_ref[1] - d0[1], diag[1] - d0[1]
    print(form, f"witness gain {gain:.4f} vs {gain_ref:.4f}, spread {diag[2]:.4f} vs {d_ref[2]:.4f}")
    assert abs(gain) > 10.0
    assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref)
    assert abs(diag[2] - d_ref[2]) <= 0.005 * d_ref[2] + 1e-3


def test_mixed64_pipelined_matches_separate_calls(wk):
    """The FP64-solve form's pipelined step (its field window in global memory) against the
    same steps taken one call at a time."""
    import torch
    cfg = synth.config_blowout(n_beam=1 << 15, nr=64, nxi=256)
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    out = []
    for pipelined in (True, False):
        with wk.Simulations([cfg], wk.WAKE_MIXED64) as s:
            wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
            wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
            if pipelined:
                wk.wake_step(s.h, 3)
            else:
                for _ in range(3):
                    wk.wake_beam_deposit(s.h)
                    wk.wake_plasma_march(s.h)
                    wk.wake_beam_push(s.h)
            assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
            out.append((s.fields(0)["ez"].cpu().numpy(), s.diagnostics()[0]))
    (ea, da), (eb, db) = out
    assert np.abs(ea - eb).max() <= 2e-3 * np.abs(eb).max()
    assert da[0] == db[0] and abs(da[1] - db[1]) <= 1e-3 * abs(db[1] - cfg.gamma_b)
