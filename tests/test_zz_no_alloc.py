"""wake_beam_deposit_noalloc (the beam deposit into a static device scratch grid, no
allocation) against the handle's wake_beam_deposit, through the C ABI.

The file sorts last so that its GPU test also runs after every other test in one process;
it passes alone in a fresh process as well (the first call does the per-device set-up).
"""
import ctypes as C

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def wk():
    from paper_1411_3246_gb300 import build, wake
    build.build()
    return wake


def test_noalloc_rejects_grids_beyond_the_scratch(wk):
    """Checked on the host before any CUDA call: runs without a GPU."""
    L = wk.lib()
    cfg = synth.config_blowout(n_beam=1 << 10, nr=1024, nxi=1024)  # 1025^2 nodes > 524288
    p = wk.params_of(cfg, wk.WAKE_FP64)
    rc = L.wake_beam_deposit_noalloc(C.byref(p), C.c_void_p(256), None, None, C.c_void_p(256))
    assert rc == wk.WAKE_EINVAL
    assert "WAKE_NOALLOC_MAX_NODES" in wk.wake_last_error()
    cfg = synth.config_blowout(n_beam=1 << 10, nr=64, nxi=128)
    p = wk.params_of(cfg, wk.WAKE_FP64)
    assert L.wake_beam_deposit_noalloc(C.byref(p), None, None, None, C.c_void_p(256)) == wk.WAKE_EINVAL
    assert L.wake_beam_deposit_noalloc(C.byref(p), C.c_void_p(256), None, None, None) == wk.WAKE_EINVAL
    assert (cfg.nr + 1) * (cfg.nxi + 1) <= wk.WAKE_NOALLOC_MAX_NODES


@pytest.mark.gpu
@pytest.mark.parametrize("steps", [0, 3])
def test_noalloc_deposit_matches_handle_deposit_two_calls(wk, steps):
    import torch
    assert torch.cuda.is_available()
    cfg = synth.config_blowout(n_beam=1 << 15, nr=64, nxi=256)
    nm_p, nm_b = synth.plasma_normals(cfg), synth.beam_normals(cfg)
    with wk.Simulations([cfg], wk.WAKE_FP64) as s:
        wk.wake_load_plasma(s.h, 0, torch.from_numpy(nm_p).cuda())
        wk.wake_load_beam(s.h, 0, torch.from_numpy(nm_b).cuda())
        if steps:
            wk.wake_step(s.h, steps)
        wk.wake_beam_deposit(s.h)
        ref = s.nb(0).cpu().numpy()
        xyz, lost = s.beam(0)
        assert s.status(0) == wk.WAKE_OK, wk.wake_last_error()
    params = wk.params_of(cfg, wk.WAKE_FP64)
    scale = np.abs(ref).max()
    assert scale > 0
    for call in range(2):
        nb = torch.full((cfg.nxi + 1, cfg.nr + 1), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        wk.wake_beam_deposit_noalloc(params, xyz, None if steps == 0 else lost, nb)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call > 0:
            assert free1 == free0, "a repeated call changed the device's free memory"
        got = nb.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-12 * scale, call
