"""Plasma-particle trapping (Sec. I: plasma particles past a threshold become beam particles
that follow the full equations of motion) through the C ABI, against the oracle's trapping run
(orc_run_trap) on the same seeded inputs.

FP64 form: the same rings are promoted at the same slices (the decision is taken in FP64 on
both sides), the promoted particles and the bunches agree to 1e-9 and the fields to 1e-8 of
their peak.  Mixed form: a ring near the threshold may be promoted a slice earlier or later,
so it is held to the blowout tolerances and to the promoted charge within 10%.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GT = 0.9  # promotes a few dozen rings per march in this warm blowout


@pytest.fixture(scope="module")
def wk():
    import torch
    from paper_1411_3246_gb300 import build, wake
    build.build()
    assert torch.cuda.is_available()
    return wake


def _case(n_beam=1 << 14):
    return synth.config_blowout(n_beam=n_beam, nr=64, nxi=256)


def _gpu(wk, cfg, prec, nsteps, gamma_t, cap):
    import torch
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    with wk.Simulations([cfg], prec) as s:
        wk.wake_set_trapping(s.h, 0, gamma_t, cap)
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        wk.wake_step(s.h, nsteps)
        xyz_t = torch.zeros((6, max(cap, 1)), dtype=torch.float64, device="cuda")
        w_t = torch.zeros(max(cap, 1), dtype=torch.float64, device="cuda")
        lost_t = torch.zeros(max(cap, 1), dtype=torch.uint8, device="cuda")
        count, dropped = wk.wake_trapped(s.h, 0, xyz_t, w_t, lost_t)
        xyz, lost = s.beam(0)
        f = {k: v.cpu().numpy() for k, v in s.fields(0).items()}
        diag = s.diagnostics()[0]
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    return {"count": count, "dropped": dropped, "xyz_t": xyz_t.cpu().numpy()[:, :count],
            "w_t": w_t.cpu().numpy()[:count], "lost_t": lost_t.cpu().numpy()[:count], "xyz": xyz.cpu().numpy(),
            "lost": lost.cpu().numpy(), "fields": f, "diag": diag}


def _oracle(cfg, nsteps, gamma_t, cap):
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    pl = oracle.plasma_init(cfg, nm_p)
    out, b, n_cur, dropped = oracle.run_trap(cfg, pl, oracle.beam_init(cfg, nm_b), nsteps, gamma_t,
                                             cfg.n_beam + cap)
    return out, b, n_cur, dropped


def test_fp64_trapping_matches_oracle(wk):
    cfg = _case()
    cap = 200
    g = _gpu(wk, cfg, wk.WAKE_FP64, 2, GT, cap)
    out, b, n_cur, dropped = _oracle(cfg, 2, GT, cap)
    n0 = cfg.n_beam
    assert g["count"] == n_cur - n0 > 10 and g["dropped"] == dropped == 0
    keys = ("x", "y", "xi", "ux", "uy", "uz")
    for row, key in enumerate(keys):
        ref = b[key][n0:n_cur]
        assert np.abs(g["xyz_t"][row] - ref).max() <= 1e-9 * max(np.abs(ref).max(), 1.0), key
    np.testing.assert_allclose(g["w_t"], b["wt"][n0:n_cur], rtol=1e-12)
    np.testing.assert_array_equal(g["lost_t"], b["lost"][n0:n_cur])
    keep = b["lost"][:n0] == 0
    np.testing.assert_array_equal(g["lost"], b["lost"][:n0])
    for row, key in enumerate(keys):
        assert np.abs(g["xyz"][row][keep] - b[key][:n0][keep]).max() <= 1e-9 * max(np.abs(b[key][:n0]).max(), 1.0)
    scale = np.abs(out["ez"]).max()
    for k in ("psi", "ez", "er", "bth"):
        assert np.abs(g["fields"][k] - out[k]).max() <= 1e-8 * scale, k


def test_mixed_trapping_close_to_oracle(wk):
    cfg = _case()
    cap = 400
    g = _gpu(wk, cfg, wk.WAKE_MIXED, 2, GT, cap)
    out, b, n_cur, _ = _oracle(cfg, 2, GT, cap)
    n0 = cfg.n_beam
    q_ref, q = b["wt"][n0:n_cur].sum(), g["w_t"].sum()
    print(f"promoted: {g['count']} vs {n_cur - n0}, charge {q:.6f} vs {q_ref:.6f}")
    assert abs(q - q_ref) <= 0.1 * q_ref
    pk_ref = np.abs(out["ez"][:, 0]).max()
    assert abs(np.abs(g["fields"]["ez"][:, 0]).max() - pk_ref) <= 0.01 * pk_ref


def test_threshold_below_every_gamma_changes_nothing(wk):
    """A threshold below every ring's Gamma (this plasma's smallest is ~0.58) promotes nothing:
    the run equals the same run without trapping."""
    import torch
    cfg = _case()
    g = _gpu(wk, cfg, wk.WAKE_FP64, 2, 0.3, 50)
    assert g["count"] == 0
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        for _ in range(2):
            wk.wake_beam_deposit(s.h)
            wk.wake_plasma_march(s.h)
            wk.wake_beam_push(s.h)
        ez = s.fields(0)["ez"].cpu().numpy()
        xyz = s.beam(0)[0].cpu().numpy()
    assert np.abs(g["fields"]["ez"] - ez).max() <= 1e-12 * np.abs(ez).max()
    assert np.abs(g["xyz"] - xyz).max() <= 1e-12 * np.abs(xyz).max()


def test_capacity_overflow_counts_dropped(wk):
    """Room for 5 promoted particles: the first 5 promotions join the beam, the rest are
    counted as dropped, as in the oracle's run with the same room (the later steps then see
    the smaller beam, on both sides)."""
    cfg = _case()
    g = _gpu(wk, cfg, wk.WAKE_FP64, 2, GT, 5)
    _, b, n_cur, dropped = _oracle(cfg, 2, GT, 5)
    assert n_cur - cfg.n_beam == 5 and dropped > 0
    assert g["count"] == 5 and g["dropped"] == dropped
    np.testing.assert_allclose(g["w_t"], b["wt"][cfg.n_beam:n_cur], rtol=1e-12)


def test_trapping_set_up_errors(wk):
    import torch
    cfg = _case()
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_beam(s.h, 0, torch.from_numpy(synth.beam_normals(cfg)).cuda())
        with pytest.raises(wk.WakeError) as e:
            wk.wake_set_trapping(s.h, 0, GT, 10)  # the beam is already loaded
        assert e.value.code == wk.WAKE_ESTATE
        with pytest.raises(wk.WakeError) as e:
            wk.wake_trapped(s.h, 0)
        assert e.value.code == wk.WAKE_ESTATE
    with wk.Simulations([cfg, cfg], wk.WAKE_FP64) as s:
        with pytest.raises(wk.WakeError) as e:
            wk.wake_set_trapping(s.h, 0, GT, 10)
        assert e.value.code == wk.WAKE_EINVAL
    frozen = synth.config_blowout(n_beam=0, nr=64, nxi=256)
    with wk.Simulations([frozen], wk.WAKE_FP64) as s:
        with pytest.raises(wk.WakeError) as e:
            wk.wake_set_trapping(s.h, 0, GT, 10)
        assert e.value.code == wk.WAKE_EINVAL
