"""Batched simulations (one handle, uneven sizes) through the C ABI: the batched deposit and
push, one march launch per tile class, the CUDA-graph step, and every compiled tile width,
each against the FP64 oracle run on every simulation alone."""
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


def small_batch():
    """Five simulations of the batched sweep's physics (linear driver + witness, warm
    plasma, seeded delays and temperatures) at test sizes."""
    shapes = [(32, 64, 2048), (48, 96, 4096), (64, 128, 3000), (96, 80, 6000), (128, 160, 8192)]
    out = []
    for cfg, (nr, nxi, nb) in zip(synth.config_batch(n_sims=len(shapes)), shapes):
        cfg.nr, cfg.nxi = nr, nxi
        out.append(synth.two_bunch(cfg, 0.3, cfg.xi_w - cfg.xi_d, nb))
    return out


def _load(wk, s, cfgs):
    """Load every simulation; the input tensors are returned so that they outlive the
    handle's (possibly separate) stream's use of them."""
    import torch
    keep = []
    for c in cfgs:
        nm = synth.plasma_normals(c)
        keep.append((None if nm is None else torch.from_numpy(nm).cuda(),
                     torch.from_numpy(synth.beam_normals(c)).cuda() if c.n_beam else None))
    torch.cuda.synchronize()  # the copies ran on torch's stream; the handle may use another
    for i, (tp, tb) in enumerate(keep):
        wk.wake_load_plasma(s.h, i, tp)
        if tb is not None:
            wk.wake_load_beam(s.h, i, tb)
    return keep


def _collect(wk, s, cfgs):
    out = []
    for i in range(len(cfgs)):
        f = {k: v.cpu().numpy() for k, v in s.fields(i).items()}
        if cfgs[i].n_beam:
            xyz, lost = s.beam(i)
            f["xyz"], f["lost"] = xyz.cpu().numpy(), lost.cpu().numpy()
        assert s.status(i) == wk.WAKE_OK, wk.wake_last_error()
        out.append(f)
    return out


def _run_batch(wk, cfgs, prec, nsteps, stream):
    with wk.Simulations(cfgs, prec, stream) as s:
        keep = _load(wk, s, cfgs)
        wk.wake_step(s.h, nsteps)
        res = _collect(wk, s, cfgs)
        del keep
        tiles = [wk.wake_tile(s.h, i) for i in range(len(cfgs))]
    return res, tiles


def _oracle_steps(cfg, nsteps):
    pl = oracle.plasma_init(cfg, synth.plasma_normals(cfg))
    bm = oracle.beam_init(cfg, synth.beam_normals(cfg))
    ref = oracle.run(cfg, pl, bm, nsteps)
    return ref, bm


def test_batched_fp64_steps_match_oracle_graph_path(wk):
    import torch
    cfgs = small_batch()
    res, tiles = _run_batch(wk, cfgs, wk.WAKE_FP64, 3, torch.cuda.Stream())
    assert all(t[0] == 512 for t in tiles)
    for cfg, got in zip(cfgs, res):
        ref, bm = _oracle_steps(cfg, 3)
        assert np.array_equal(got["lost"], bm["lost"])
        keep = bm["lost"] == 0
        for row, key in enumerate(("x", "y", "xi", "ux", "uy", "uz")):
            a, b = got["xyz"][row][keep], bm[key][keep]
            assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1.0), key
        scale = np.abs(ref["ez"]).max()
        for k in ("psi", "ez", "er", "bth"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-8 * scale, k


def test_batched_graph_and_direct_launches_agree(wk):
    import torch
    cfgs = small_batch()[:3]
    g, _ = _run_batch(wk, cfgs, wk.WAKE_FP64, 4, torch.cuda.Stream())
    d, _ = _run_batch(wk, cfgs, wk.WAKE_FP64, 4, None)  # legacy default stream: no graph
    for a, b in zip(g, d):
        assert np.array_equal(a["lost"], b["lost"])
        for k in ("psi", "ez", "er", "bth"):
            assert np.abs(a[k] - b[k]).max() <= 1e-10 * np.abs(b["ez"]).max(), k
        keep = b["lost"] == 0
        assert np.abs(a["xyz"][:, keep] - b["xyz"][:, keep]).max() <= 1e-10 * np.abs(b["xyz"][:, keep]).max()


@pytest.mark.parametrize("nt", [128, 256, 512])
def test_mixed_tile_widths_match_oracle_linear(wk, nt, monkeypatch):
    """Each compiled tile width of the mixed march: linear frozen-driver fields within 1e-5 of
    peak |E_z| of the FP64 oracle."""
    monkeypatch.setenv("WAKE_TILE_NT", str(nt))
    cfgs = [synth.config_linear(nr=128, nxi=256), synth.config_linear(nr=96, nxi=200, n0=0.05)]
    with wk.Simulations(cfgs, wk.WAKE_MIXED) as s:
        keep = _load(wk, s, cfgs)
        wk.wake_plasma_march(s.h)
        res = _collect(wk, s, cfgs)
        del keep
        tiles = [wk.wake_tile(s.h, i) for i in range(len(cfgs))]
    assert all(t[0] == nt for t in tiles), tiles
    for cfg, got in zip(cfgs, res):
        ref = oracle.march(cfg, oracle.plasma_init(cfg, None), oracle.nb_analytic(cfg))
        scale = np.abs(ref["ez"]).max()
        for k in ("psi", "ez", "er", "bth"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-5 * scale, (nt, k)


def test_batched_mixed_autotuned_steps_match_oracle(wk, monkeypatch):
    """Autotuned tiles, graph path, mixed form: witness mean energy gain within 0.5% and
    fields within 1e-4 of peak |E_z| (warm plasma) of the FP64 oracle."""
    import torch
    monkeypatch.setenv("WAKE_BATCH_PIPELINE", "0")
    cfgs = small_batch()
    for c in cfgs:
        c.ds = 50.0
    with wk.Simulations(cfgs, wk.WAKE_MIXED, torch.cuda.Stream()) as s:
        keep = _load(wk, s, cfgs)
        d0 = s.diagnostics()
        wk.wake_step(s.h, 3)
        res = _collect(wk, s, cfgs)
        d1 = s.diagnostics()
        tiles = [wk.wake_tile(s.h, i) for i in range(len(cfgs))]
        del keep
    assert all(t[0] in (128, 256, 512) and t[1] >= 1 for t in tiles)
    for i, cfg in enumerate(cfgs):
        ref, bm = _oracle_steps(cfg, 3)
        dr = oracle.diagnostics(cfg, bm)
        gain, gain_ref = d1[i][1] - d0[i][1], dr[1] - d0[i][1]
        assert abs(gain_ref) > 0.01
        assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref), (i, gain, gain_ref)
        scale = np.abs(ref["ez"]).max()
        assert np.abs(res[i]["ez"] - ref["ez"]).max() <= 1e-4 * scale, i


def _mixed_batch_run(wk, cfgs, nsteps):
    import torch
    with wk.Simulations(cfgs, wk.WAKE_MIXED, torch.cuda.Stream()) as s:
        keep = _load(wk, s, cfgs)
        d0 = s.diagnostics()
        wk.wake_step(s.h, nsteps)
        kern_ms = wk.wake_step_kernel_ms(s.h)
        res = _collect(wk, s, cfgs)
        d1 = s.diagnostics()
        del keep
    return d0, d1, res, kern_ms


def test_batched_pipelined_steps_match_oracle_and_graph_path(wk, monkeypatch):
    """Mixed form, one persistent launch of every simulation's pipelined steps (the default
    for a mixed handle whose simulations all have beams): witness energy gain within 0.5% and
    fields within 1e-4 of peak |E_z| of the FP64 oracle, and the graph path's results within
    FP32 rounding."""
    cfgs = small_batch()
    for c in cfgs:
        c.ds = 50.0
    d0, d1, res, kern_ms = _mixed_batch_run(wk, cfgs, 3)
    assert kern_ms > 0.0  # the pipelined launch ran
    monkeypatch.setenv("WAKE_BATCH_PIPELINE", "0")
    _, g1, gres, gms = _mixed_batch_run(wk, cfgs, 3)
    assert gms == 0.0  # the graph path launches no pipelined kernel
    for i, cfg in enumerate(cfgs):
        ref, bm = _oracle_steps(cfg, 3)
        dr = oracle.diagnostics(cfg, bm)
        gain, gain_ref = d1[i][1] - d0[i][1], dr[1] - d0[i][1]
        assert abs(gain - gain_ref) <= 0.005 * abs(gain_ref), (i, gain, gain_ref)
        scale = np.abs(ref["ez"]).max()
        assert np.abs(res[i]["ez"] - ref["ez"]).max() <= 1e-4 * scale, i
        assert np.array_equal(res[i]["lost"], gres[i]["lost"])
        assert np.abs(res[i]["ez"] - gres[i]["ez"]).max() <= 1e-4 * scale, i
        assert abs((d1[i][1] - g1[i][1])) <= 1e-3 * abs(gain_ref) + 1e-6 * cfg.gamma_b, i
