"""Benchmark: plasma pushes/s of the quasi-static wake method on the blowout two-bunch workload.

Workload: warm plasma u_th = 0.01, Nr = 512 over 8 k_p^-1, Nxi = 2048 over 12 k_p^-1, 8 rings
per cell (4096 rings per slice), two-bunch Eq. 12 driver n_b/n_p = 8, sigma_r = 0.2,
sigma_z = 0.6, gamma = 4e4, witness 4.5 behind with 30% of the drive charge, 1,048,576 beam
macroparticles, 200 beam steps of ds = 5.  One bench step is one run of that workload from
its initial beam: 200 x (beam deposit -> xi-march -> beam push), i.e. 200 x 4096 x 2049
plasma pushes and 200 x 1,048,576 beam pushes, taken by one wake_step(200) call (pipelined:
one cooperative launch, one beam step per SM).

Arms:
  default           the library's mixed-precision form (FP32 rings and fields, wide sums)
  --impl reference  the FP64 CPU oracle on the host cores (bounded sample of the same steps)

Timing: W untimed warm-up runs, then K runs, each bracketed by CUDA events on the library's
stream; before each timed run the beam is re-initialised on the device (outside the timed
region) and a 512 MB buffer is written to flush L2.  The JSON line also carries the plain
FP64 GPU path (same scheme, FP64 throughout), an end-to-end number through the C ABI from
pinned host buffers, the step kernel's roofline and the oracle CPU baseline, and further
legs (each skippable by its flag): the batched sweep, the adjoint, the large configuration,
the Table I beam carried 1.49 m and the single bunch of the OSIRIS parameter set carried
1.4 m.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

# Algorithmic FP32 operations (an FMA counts 2, a divide or square root 1, a hat deposit two
# nodes per value): per plasma push (one ring advanced one slice: stage-1 ring quantities and
# current deposits 66, the move to the midpoint and its charge 51, stage 2 63, the full step and
# its charge 70), per grid node and field stage (the radial solves, a Thomas-equivalent count),
# and per beam push (bilinear gather, Boris step, deposit into the next step's grid).
FLOP_PER_PUSH = 250.0
FLOP_PER_NODE_STAGE = 62.0
FLOP_PER_BEAM_PUSH = 140.0
BEAM_STEPS = 200
# DRAM traffic of one launch of the step kernel on this workload (200 steps), from one ncu
# capture with one pass (dram__bytes_read.sum + dram__bytes_write.sum: 950.72 + 149.46 MB),
# valid while the kernel's sources hash to STEP_TRAFFIC_SOURCES
STEP_TRAFFIC_BYTES = 1100.18e6
STEP_TRAFFIC_SOURCES = "f9ea6843b093240b"
STEP_SOURCES = ("beam.cuh", "march.cuh", "march_mixed.cu", "march_wide.cuh", "pipeline.cuh", "wake_common.cuh")


def step_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1411_3246_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
# kernels of one pipelined wake_step launch sequence: slip bound, three of the cell sort,
# deposit and normalise of the first step's density, the step kernel
KERNELS_PER_RUN = 7


def workload():
    return synth.config_blowout(n_beam=1 << 20)


def plasma_pushes_per_step(cfg):
    """Plasma pushes of one march: every ring through every slice xi_0 .. xi_Nxi."""
    return cfg.nr * cfg.ppc * (cfg.nxi + 1)


def march_flops(cfg):
    return plasma_pushes_per_step(cfg) * FLOP_PER_PUSH + 2 * (cfg.nxi + 1) * (cfg.nr + 1) * FLOP_PER_NODE_STAGE


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz):
    # nominal: 152 SMs x 128 FP32 lanes x 2 flop (FMA) per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fma_peak_leg(local):
    """The ALU peaks measured on this GPU in this run: FP32 and FP64 FMA throughput of the
    package's micro-benchmark (16 independent FMA chains per thread, 8 CTAs of 256 threads per
    SM, CUDA events), with the SM clock sampled while it runs."""
    from paper_1411_3246_gb300 import build, peak
    build.build_peak()
    peak.fma_tflops(False, iters=1 << 12)  # warm-up (module load, clocks up)
    with ClockSampler(local) as clk:
        f32, ms32, _ = peak.fma_tflops(False)
        f64, ms64, _ = peak.fma_tflops(True)
    c = clk.summary()
    return {"fp32_tflops": f32, "fp64_tflops": f64, "fp32_ms": ms32, "fp64_ms": ms64, "clocks": c,
            "fp32_nominal_at_max_clock": fp32_peak_tflops(2070.0),
            "how": "FMA chains (16 per thread, 256-thread CTAs, 8 per SM), an FMA = 2 flop, CUDA events"}


def latency_leg(wake, torch, stream, nrep=20):
    """The frozen-driver linear workload (Nr=128 over 6, Nxi=256 over 10, 4 rings/cell, cold,
    n_b/n_p = 0.1): microseconds per xi-march (one CTA marches the whole box), FP64 and mixed,
    averaged over nrep back-to-back marches after two untimed ones (CUDA events)."""
    cfg = synth.config_linear()
    out = {}
    for name, prec in (("fp64", wake.WAKE_FP64), ("mixed", wake.WAKE_MIXED)):
        sim = wake.Simulations([cfg], prec, stream)
        with torch.cuda.stream(stream):
            wake.wake_load_plasma(sim.h, 0, None)
            for _ in range(2):
                wake.wake_plasma_march(sim.h)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(nrep):
                wake.wake_plasma_march(sim.h)
            ev[1].record(stream)
        stream.synchronize()
        st = sim.status(0)
        sim.close()
        if st != wake.WAKE_OK:
            raise RuntimeError(f"latency leg: status {st}")
        us = 1e3 * ev[0].elapsed_time(ev[1]) / nrep
        out[name] = {"us_per_march": us, "plasma_pushes_per_s": plasma_pushes_per_step(cfg) / (us * 1e-6)}
    out["workload"] = (f"linear frozen driver, Nr={cfg.nr} x Nxi={cfg.nxi}, {cfg.ppc} rings/cell, cold, one march "
                       f"({plasma_pushes_per_step(cfg)} plasma pushes), {nrep} marches averaged")
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier_max(x, world):
    """The largest x over the ranks (each rank's timed region ends at its own clock; the job's
    time is the slowest rank's).  NCCL reduces a CUDA tensor, gloo a host one."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base, rank):
    """Seed of rank's replica: the replicas are independent simulations of the same workload."""
    return base + 1000 * rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_step_rate(cfg, nsteps):
    """The FP64 oracle, as it stands, on nsteps full beam steps of the workload (one host
    thread).  Returns seconds per step."""
    import oracle
    pl = oracle.plasma_init(cfg, synth.plasma_normals(cfg))
    bm = oracle.beam_init(cfg, synth.beam_normals(cfg))
    t = time.perf_counter()
    oracle.run(cfg, pl, bm, nsteps)
    return (time.perf_counter() - t) / nsteps


_ORC = None


def _orc_init(cfg):
    """Worker set-up of the parallel oracle: the workload's plasma and beam (each worker one
    independent copy of the same simulation)."""
    global _ORC
    import oracle
    _ORC = (cfg, oracle.plasma_init(cfg, synth.plasma_normals(cfg)), oracle.beam_init(cfg, synth.beam_normals(cfg)))


def _orc_step(_):
    """One beam step (deposit, march, push) of the worker's copy; returns its seconds."""
    import oracle
    cfg, pl, bm = _ORC
    t = time.perf_counter()
    oracle.run(cfg, pl, bm, 1)
    return time.perf_counter() - t


class OraclePool:
    """The FP64 oracle, as it stands, on the host's cores: one worker process per core (spawned,
    never forked from a process that has touched the GPU), each advancing its own copy of the
    workload one beam step per task.  A round is one step on every worker at once."""

    def __init__(self, cfg, procs=None):
        import multiprocessing as mp

        import oracle
        oracle.build()
        self.procs = procs or len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_orc_init, initargs=(cfg,))

    def round(self):
        """Wall seconds of one step on every worker."""
        t = time.perf_counter()
        self.pool.map(_orc_step, range(self.procs), chunksize=1)
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, world, rank):
    """--impl reference: the oracle on the host cores, same metric and workload.  Each bench
    step is one beam step of the workload on every core at once (one independent copy per
    core); the value is the plasma pushes of all copies over the wall time."""
    if rank != 0:
        return
    cfg = workload()
    pool = OraclePool(cfg)
    for _ in range(args.warmup):
        pool.round()
    times = [pool.round() for _ in range(args.steps)]
    pool.close()
    tot = sum(times)
    v = plasma_pushes_per_step(cfg) * pool.procs * args.steps / tot
    line = {"impl": "reference", "metric": "plasma_pushes_per_s", "value": v, "unit": "pushes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(cfg, world, BEAM_STEPS),
            "cpu_baseline": {"value": v, "unit": "pushes/s", "cores": pool.procs, "kind": "oracle",
                             "sample": f"each step: one beam step (deposit, march, push) of the workload's "
                                       f"{BEAM_STEPS} on each of {pool.procs} processes at once (one "
                                       f"independent copy per core), FP64 oracle"},
            "e2e": {"value": v, "unit": "pushes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(cfg, world, beam_steps):
    return {"workload": f"blowout two-bunch warm plasma, Nr={cfg.nr} x Nxi={cfg.nxi}, {cfg.ppc} rings/cell, "
                        f"{cfg.n_beam} beam particles, {beam_steps} beam steps of ds={cfg.ds:g}",
            "step": f"one run of the workload from its initial beam: {beam_steps} x (deposit, xi-march, push)",
            "nr": cfg.nr, "nxi": cfg.nxi, "ppc": cfg.ppc, "n_beam": cfg.n_beam, "u_th": cfg.u_th,
            "beam_steps": beam_steps, "plasma_pushes_per_step": plasma_pushes_per_step(cfg) * beam_steps,
            "beam_pushes_per_step": cfg.n_beam * beam_steps,
            "l2": "flushed before each timed run (512 MB write); the run's working set exceeds L2",
            "parallelism": f"replicas x{world}"}


def batched_leg(wake, torch, n_sims, nsteps, rank, flush, world):
    """The batched sweep: n_sims simulations of uneven size, temperature and witness delay in
    one handle (mixed form), nsteps beam steps by one wake_step call (every simulation's steps
    pipelined in one persistent launch).  One untimed run (allocation), then one timed run
    from the initial beams."""
    cfgs = synth.config_batch(n_sims=n_sims, n_steps=nsteps, seed=replica_seed(synth.SEED_BASE + 3, rank))
    stream = torch.cuda.Stream()
    pl = [synth.plasma_normals(c) for c in cfgs]
    bm = [synth.beam_normals(c) for c in cfgs]
    sim = wake.Simulations(cfgs, wake.WAKE_MIXED, stream)
    with torch.cuda.stream(stream):
        dpl = [None if a is None else torch.from_numpy(a).to("cuda", non_blocking=False) for a in pl]
        dbm = [torch.from_numpy(a).to("cuda", non_blocking=False) for a in bm]
        for i in range(n_sims):
            wake.wake_load_plasma(sim.h, i, dpl[i])
        times = []
        for run in range(2):
            for i in range(n_sims):
                wake.wake_load_beam(sim.h, i, dbm[i])
            flush.fill_(1)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            wake.wake_step(sim.h, nsteps)
            ev[1].record(stream)
            stream.synchronize()
            times.append(ev[0].elapsed_time(ev[1]))
    st = [sim.status(i) for i in range(n_sims)]
    sim.close()
    if any(x != wake.WAKE_OK for x in st):
        raise RuntimeError(f"batched leg: simulation status {st}")
    pushes = sum(c.nr * c.ppc * (c.nxi + 1) for c in cfgs) * nsteps
    t = barrier_max(times[-1] / 1e3, world)
    return {"value": world * pushes / t, "unit": "pushes/s", "ms_per_run": 1e3 * t, "sims": n_sims,
            "beam_steps": nsteps, "plasma_pushes_per_run": pushes,
            "beam_pushes_per_run": sum(c.n_beam for c in cfgs) * nsteps,
            "beam_pushes_per_s": world * sum(c.n_beam for c in cfgs) * nsteps / t,
            "first_run_ms": times[0],
            "workload": "batched sweep: Nr in {128..1024}, Nxi in {512..4096} log-uniform, ppc 4, "
                        "u_th ~ U[0,0.02], witness delay ~ U[3.5,5.5], 64k-256k beam particles each",
            "dtype": "f32",
            "form": ("one CUDA graph per beam step: batched deposit, one march launch per tile class, "
                     "batched push (WAKE_BATCH_PIPELINE=0)" if os.environ.get("WAKE_BATCH_PIPELINE", "1") == "0"
                     else "every simulation's steps pipelined in one persistent launch (wide march, "
                          "256-thread CTAs, two per SM); WAKE_BATCH_PIPELINE=0 takes the CUDA-graph step")}


def large_leg(wake, torch, nsteps, rank, flush, world):
    """The large configuration (mixed, the wide march form): one run of nsteps beam steps from
    the initial beam by one wake_step call, after an untimed run of one step (allocation)."""
    cfg = synth.config_large()
    cfg.seed = replica_seed(cfg.seed, rank)
    stream = torch.cuda.Stream()
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).pin_memory()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
    with torch.cuda.stream(stream):
        dp, db = nm_p.cuda(non_blocking=True), nm_b.cuda(non_blocking=True)
        wake.wake_load_plasma(sim.h, 0, dp)
        wake.wake_load_beam(sim.h, 0, db)
        wake.wake_step(sim.h, 1)
        wake.wake_load_beam(sim.h, 0, db)
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wake.wake_step(sim.h, nsteps)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    st = sim.status(0)
    sim.close()
    if st != wake.WAKE_OK:
        raise RuntimeError(f"large leg: simulation status {st}: {wake.wake_last_error()}")
    pushes = plasma_pushes_per_step(cfg) * nsteps
    t = barrier_max(ms / 1e3, world)
    return {"value": world * pushes / t, "unit": "pushes/s", "ms_per_run": 1e3 * t, "beam_steps": nsteps,
            "beam_pushes_per_s": world * cfg.n_beam * nsteps / t,
            "workload": f"large: Nr={cfg.nr} x Nxi={cfg.nxi}, {cfg.ppc} rings/cell ({cfg.nr * cfg.ppc} per slice), "
                        f"u_th={cfg.u_th}, {cfg.n_beam} beam particles, {nsteps} of the configuration's 1000 steps",
            "form": "wide march (rings in global memory, chunks of 512 x 8 slots), pipelined", "dtype": "f32"}


def large_fp64_leg(wake, torch, nsteps, nslices, rank, world):
    """The plain FP64 path on the large configuration, a bounded sample: its radial grid,
    plasma (Nr=2048, 65,536 rings per slice, u_th=0.02) and two-bunch beam over the whole box,
    cut into nslices slices instead of 8192 (the per-slice work of the march is the same), 2^20
    beam particles, nsteps pipelined steps after one untimed step.  The FP64 wide form keeps
    its node arrays in global memory; the whole configuration would take hours."""
    cfg = synth.config_large(n_beam=1 << 20)
    cfg.seed = replica_seed(cfg.seed, rank)
    cfg.nxi = nslices
    stream = torch.cuda.Stream()
    sim = wake.Simulations([cfg], wake.WAKE_FP64, stream)
    with torch.cuda.stream(stream):
        dp = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
        db = torch.from_numpy(synth.beam_normals(cfg)).cuda()
        wake.wake_load_plasma(sim.h, 0, dp)
        wake.wake_load_beam(sim.h, 0, db)
        wake.wake_step(sim.h, 1)
        wake.wake_load_beam(sim.h, 0, db)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wake.wake_step(sim.h, nsteps)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    st = sim.status(0)
    sim.close()
    if st != wake.WAKE_OK:
        raise RuntimeError(f"large FP64 leg: simulation status {st}: {wake.wake_last_error()}")
    pushes = plasma_pushes_per_step(cfg) * nsteps
    t = barrier_max(ms / 1e3, world)
    return {"value": world * pushes / t, "unit": "pushes/s", "ms_per_run": 1e3 * t, "beam_steps": nsteps,
            "workload": f"the large configuration's radial grid, plasma (Nr={cfg.nr}, {cfg.nr * cfg.ppc} rings per "
                        f"slice) and beam over its whole box in {nslices} slices (the configuration has 8192), 2^20 "
                        f"beam particles, {nsteps} pipelined steps", "dtype": "f64",
            "form": "FP64 wide march: rings and node arrays in global memory"}


def facet_leg(wake, torch, length_m, rank, flush, world):
    """The Table I two-bunch beam (2^20 particles, zero emittance) carried length_m metres
    through a 5 eV plasma (Nr=256 over 6, Nxi=1024 over 16, 8 rings/cell): one wake_step call
    of all its steps, timed, after an untimed step; then the witness spectrum."""
    from paper_1411_3246_gb300 import studies
    cfg = synth.config_facet(te_ev=5.0)
    cfg.seed = replica_seed(cfg.seed, rank)
    nsteps = studies.steps_for_length(length_m, cfg.ds)
    stream = torch.cuda.Stream()
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).pin_memory()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
    with torch.cuda.stream(stream):
        dp, db = nm_p.cuda(non_blocking=True), nm_b.cuda(non_blocking=True)
        wake.wake_load_plasma(sim.h, 0, dp)
        wake.wake_load_beam(sim.h, 0, db)
        wake.wake_step(sim.h, 1)
        wake.wake_load_beam(sim.h, 0, db)
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wake.wake_step(sim.h, nsteps)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    xyz, lost = sim.beam(0)
    torch.cuda.synchronize()
    e = studies.witness_energies_gev(xyz.cpu().numpy(), lost.cpu().numpy(), cfg.n_drive)
    st = sim.status(0)
    sim.close()
    if st != wake.WAKE_OK:
        raise RuntimeError(f"facet leg: simulation status {st}: {wake.wake_last_error()}")
    pushes = plasma_pushes_per_step(cfg) * nsteps
    t = barrier_max(ms / 1e3, world)
    return {"value": world * pushes / t, "unit": "pushes/s", "ms_per_run": 1e3 * t, "beam_steps": nsteps,
            "beam_pushes_per_s": world * cfg.n_beam * nsteps / t,
            "witness_peak_gev": studies.spectrum_peak(e), "witness_mean_gev": float(e.mean()),
            "workload": f"Table I two-bunch beam, {cfg.n_beam} particles, carried {length_m} m "
                        f"({nsteps} steps of ds={cfg.ds}) in a 5 eV plasma, Nr={cfg.nr} x Nxi={cfg.nxi}, "
                        f"{cfg.ppc} rings/cell", "dtype": "f32"}


def osiris_leg(wake, torch, length_m, rank, flush, world):
    """The single-bunch parameter set of the paper's OSIRIS comparison (200 x 500 cells, 9
    rings/cell, 2.5e6 beam particles) carried length_m metres (k_p^-1 = 0.367 mm): one
    wake_step call of all its steps, timed, after an untimed step."""
    cfg = synth.config_osiris()
    cfg.seed = replica_seed(cfg.seed, rank)
    nsteps = int(round(length_m / 0.367e-3 / cfg.ds))
    stream = torch.cuda.Stream()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
    with torch.cuda.stream(stream):
        db = nm_b.cuda(non_blocking=True)
        wake.wake_load_plasma(sim.h, 0, None)
        wake.wake_load_beam(sim.h, 0, db)
        wake.wake_step(sim.h, 1)
        wake.wake_load_beam(sim.h, 0, db)
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wake.wake_step(sim.h, nsteps)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    d = sim.diagnostics()[0]
    st = sim.status(0)
    sim.close()
    if st != wake.WAKE_OK:
        raise RuntimeError(f"osiris leg: simulation status {st}: {wake.wake_last_error()}")
    pushes = plasma_pushes_per_step(cfg) * nsteps
    t = barrier_max(ms / 1e3, world)
    return {"value": world * pushes / t, "unit": "pushes/s", "ms_per_run": 1e3 * t, "beam_steps": nsteps,
            "beam_pushes_per_s": world * cfg.n_beam * nsteps / t, "drive_mean_gamma": d[4],
            "workload": f"single bunch of the OSIRIS comparison, {cfg.n_beam} particles, carried {length_m} m "
                        f"({nsteps} steps of ds={cfg.ds}), cold plasma, Nr={cfg.nr} x Nxi={cfg.nxi}, "
                        f"{cfg.ppc} rings/cell", "dtype": "f32"}


def slab_leg(wake, torch, nsteps, rank, flush, world):
    """The blowout workload in slab geometry (Sec. I: WAKE handles slab as well as cylindrical
    geometry): Nr=512 x Nxi=2048, 8 sheets/cell, two sheet bunches of 2^20 particles, mixed
    form, one pipelined wake_step of nsteps, timed, after an untimed step."""
    cfg = synth.config_slab_blowout(n_steps=nsteps)
    cfg.seed = replica_seed(cfg.seed, rank)
    stream = torch.cuda.Stream()
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).pin_memory()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
    with torch.cuda.stream(stream):
        dp, db = nm_p.cuda(non_blocking=True), nm_b.cuda(non_blocking=True)
        wake.wake_load_plasma(sim.h, 0, dp)
        wake.wake_load_beam(sim.h, 0, db)
        wake.wake_step(sim.h, 1)
        wake.wake_load_beam(sim.h, 0, db)
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        wake.wake_step(sim.h, nsteps)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    d = sim.diagnostics()[0]
    st = sim.status(0)
    sim.close()
    if st != wake.WAKE_OK:
        raise RuntimeError(f"slab leg: simulation status {st}: {wake.wake_last_error()}")
    t = barrier_max(ms / 1e3, world)
    return {"value": world * plasma_pushes_per_step(cfg) * nsteps / t, "unit": "pushes/s", "ms_per_run": 1e3 * t,
            "beam_steps": nsteps, "beam_pushes_per_s": world * cfg.n_beam * nsteps / t,
            "witness_mean_gamma": d[1], "workload": f"slab blowout: two sheet bunches, {cfg.n_beam} particles, "
            f"Nr={cfg.nr} x Nxi={cfg.nxi}, {cfg.ppc} sheets/cell, warm (u_th={cfg.u_th}), {nsteps} steps",
            "dtype": "f32"}


def adjoint_case(nsteps, rank):
    """The differentiation workload (synth.config_adjoint): the linear-driver grid (Nr=128 over
    6, 4 rings/cell) at Nxi=1024 over 10, two bunches, 262,144 beam particles, u_th = 0.005;
    the bench adds a 64-bin witness profile."""
    return synth.config_adjoint(nsteps, seed=replica_seed(synth.SEED_BASE + 4, rank))


def adjoint_leg(wake, torch, nsteps, rank, world):
    """One forward (observables) and one backward (gradient of both observables' sum) of the
    adjoint form on the differentiation workload, timed on the host around the synchronous
    calls."""
    cfg = adjoint_case(nsteps, rank)
    nbins = 64
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).cuda()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).cuda()
    theta = [cfg.n_w, cfg.xi_w - cfg.xi_d, cfg.sigma_zd, cfg.u_th]
    torch.cuda.synchronize()
    with wake.Adjoint(cfg, nsteps, nbins, nm_p, nm_b) as a:
        t0 = time.perf_counter()
        obs = a.forward(theta, [1.0] * nbins)
        t1 = time.perf_counter()
        g = a.backward([1.0, 1.0])
        t2 = time.perf_counter()
    fwd = barrier_max(t1 - t0, world)
    bwd = barrier_max(t2 - t1, world)
    pushes = cfg.nr * cfg.ppc * (cfg.nxi + 1) * nsteps
    # the library's plain FP64 path on the same workload (wake_step, pipelined), for comparison
    sim = wake.Simulations([cfg], wake.WAKE_FP64)
    wake.wake_load_plasma(sim.h, 0, nm_p)
    wake.wake_load_beam(sim.h, 0, nm_b)
    wake.wake_step(sim.h, 1)
    wake.wake_load_beam(sim.h, 0, nm_b)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    wake.wake_step(sim.h, nsteps)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    sim.close()
    plain = barrier_max(t4 - t3, world)
    return {"adjoint_over_forward": bwd / fwd, "forward_s": fwd, "backward_s": bwd,
            "forward_plasma_pushes_per_s": world * pushes / fwd,
            "fp64_step_plasma_pushes_per_s": world * pushes / plain, "fp64_step_s": plain, "dtype": "f64",
            "workload": f"Nr={cfg.nr} x Nxi={cfg.nxi}, {cfg.ppc} rings/cell, {cfg.n_beam} beam particles, "
                        f"{nsteps} beam steps, gradients w.r.t. n_w, delay, sigma_zd, u_th and {nbins} profile bins",
            "observables": obs, "grad_scalars": g[:4],
            "tape": "every slice's intermediates kept by the forward when they fit a quarter of the free device "
                    "memory (this workload: ~12.8 GB), else the ring state every round(sqrt(Nxi+1)) slices, "
                    "recomputed by the reverse; beam, density and fields of every step",
            "form": "pipelined: one CTA per beam step, each a few slices behind the previous (forward) or the "
                    "next (reverse) step"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed runs of the FP64 form (0: skip)")
    ap.add_argument("--mixed64-steps", type=int, default=1, help="timed runs of the FP64-solve split (0: skip)")
    ap.add_argument("--beam-steps", type=int, default=BEAM_STEPS, help="beam steps per run (profiling)")
    ap.add_argument("--nr", type=int, default=0, help="override Nr (profiling a smaller case)")
    ap.add_argument("--nxi", type=int, default=0, help="override Nxi (profiling a smaller case)")
    ap.add_argument("--n-beam", type=int, default=0, help="override the beam size (profiling)")
    ap.add_argument("--batch-sims", type=int, default=256, help="simulations of the batched leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=50, help="beam steps of the batched leg")
    ap.add_argument("--adjoint-steps", type=int, default=100, help="beam steps of the adjoint leg (0: skip)")
    ap.add_argument("--large-steps", type=int, default=304,
                    help="beam steps of the large-configuration leg (0: skip; the configuration has 1000)")
    ap.add_argument("--large-fp64-steps", type=int, default=152,
                    help="pipelined FP64 steps of the large configuration's first 256 slices (0: skip)")
    ap.add_argument("--facet-m", type=float, default=1.49,
                    help="metres the Table I beam is carried in the propagation leg (0: skip)")
    ap.add_argument("--osiris-m", type=float, default=1.4,
                    help="metres the single bunch of the OSIRIS parameter set is carried (0: skip)")
    ap.add_argument("--latency", type=int, default=1, help="time the one-march latency case (0: skip)")
    ap.add_argument("--slab-steps", type=int, default=200, help="beam steps of the slab-geometry leg (0: skip)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1411_3246_gb300 import wake
    torch.cuda.set_device(local)
    cfg = workload()
    if args.nr:
        cfg.nr = args.nr
    if args.nxi:
        cfg.nxi = args.nxi
    if args.n_beam:
        cfg = synth.two_bunch(cfg, 0.3, 4.5, args.n_beam)
    nbs = args.beam_steps
    cfg.seed = replica_seed(cfg.seed, rank)  # independent replicas
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).pin_memory()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pushes = plasma_pushes_per_step(cfg) * nbs

    def timed_runs(prec, k, w):
        """k timed runs (w untimed first) of the workload; returns per-run wall ms (events around
        wake_step), the step kernel's ms per run, and the last run's diagnostics."""
        sim = wake.Simulations([cfg], prec, stream)
        with torch.cuda.stream(stream):
            dp = nm_p.cuda(non_blocking=True)
            db = nm_b.cuda(non_blocking=True)
            wake.wake_load_plasma(sim.h, 0, dp)
        run_ms, kern_ms, diag = [], [], None
        for i in range(w + k):
            with torch.cuda.stream(stream):
                wake.wake_load_beam(sim.h, 0, db)
                flush.fill_(1)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(stream)
                wake.wake_step(sim.h, nbs)
                ev[1].record(stream)
            stream.synchronize()
            if i >= w:
                run_ms.append(ev[0].elapsed_time(ev[1]))
                kern_ms.append(wake.wake_step_kernel_ms(sim.h))
        st = sim.status(0)
        diag = sim.diagnostics()[0]
        sim.close()
        if st != wake.WAKE_OK:
            raise RuntimeError(f"simulation status {st}: {wake.wake_last_error()}")
        return run_ms, kern_ms, diag

    # --- mixed-precision arm (the headline) ---
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        run_ms, kern_ms, diag = timed_runs(wake.WAKE_MIXED, args.steps, args.warmup)
        torch.cuda.synchronize()
    barrier(world)
    clocks = clk.summary()
    tot_s = barrier_max(sum(run_ms) / 1e3, world)
    value = world * pushes * args.steps / tot_s

    # --- plain FP64 GPU path, same workload and scheme ---
    fp64 = None
    if args.fp64_steps > 0:
        r64, k64, _ = timed_runs(wake.WAKE_FP64, args.fp64_steps, 1)
        t64 = barrier_max(sum(r64) / 1e3, world)
        fp64 = {"value": world * pushes * args.fp64_steps / t64, "unit": "pushes/s",
                "ms_per_step": 1e3 * t64 / args.fp64_steps, "steps": args.fp64_steps,
                "note": "FP64 form of the same pipelined path (rings, fields and sums in FP64)"}

    # --- the precision split with FP64 sums across rings, scans and tridiagonal solves ---
    mixed64 = None
    if args.mixed64_steps > 0:
        r2, k2, d2 = timed_runs(wake.WAKE_MIXED64, args.mixed64_steps, 1)
        t2 = barrier_max(sum(r2) / 1e3, world)
        mixed64 = {"value": world * pushes * args.mixed64_steps / t2, "unit": "pushes/s",
                   "ms_per_step": 1e3 * t2 / args.mixed64_steps, "steps": args.mixed64_steps,
                   "kernel_ms": sum(k2) / len(k2), "cost_vs_mixed": (sum(r2) / len(r2)) / (sum(run_ms) / len(run_ms)),
                   "witness": {"mean_gamma": d2[1], "rms_gamma": d2[2], "alive": d2[0]},
                   "note": "WAKE_MIXED64: FP32 particle arithmetic; FP64 sums across rings, node arrays, scans and "
                           "tridiagonal solve (charge in exact fixed point); same pipelined path, field window in "
                           "global memory"}

    # --- end to end through the C ABI from pinned host buffers, one run per step ---
    e2e_steps = max(1, min(args.steps, 3))
    h2d = nm_p.numel() * 8 + nm_b.numel() * 8
    sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
    e2e_ms = []
    for i in range(e2e_steps + 1):  # the first run allocates the pipeline's grids: untimed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            dp = nm_p.cuda(non_blocking=True)
            db = nm_b.cuda(non_blocking=True)
            wake.wake_load_plasma(sim.h, 0, dp)
            wake.wake_load_beam(sim.h, 0, db)
            wake.wake_step(sim.h, nbs)
        sim.diagnostics()  # synchronous device -> host read of the run's result
        if i > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    sim.close()
    e2e_s = barrier_max(sum(e2e_ms) / 1e3, world)

    # --- batched sweep: uneven simulations in one handle, autotuned tiles, CUDA-graph steps ---
    batched = None
    if args.batch_sims > 0:
        batched = batched_leg(wake, torch, args.batch_sims, args.batch_steps, rank, flush, world)

    # --- adjoint form: gradient of the witness observables, backward / forward time ---
    adjoint = None
    if args.adjoint_steps > 0:
        adjoint = adjoint_leg(wake, torch, args.adjoint_steps, rank, world)

    # --- large configuration: Nr=2048, 65,536 rings per slice, 16M beam particles ---
    large = None
    if args.large_steps > 0:
        large = large_leg(wake, torch, args.large_steps, rank, flush, world)

    large_fp64 = None
    if args.large_fp64_steps > 0:
        large_fp64 = large_fp64_leg(wake, torch, args.large_fp64_steps, 256, rank, world)

    # --- propagation: the Table I beam carried 1.49 m (the paper's FACET run) ---
    facet = None
    if args.facet_m > 0:
        facet = facet_leg(wake, torch, args.facet_m, rank, flush, world)

    osiris = None
    if args.osiris_m > 0:
        osiris = osiris_leg(wake, torch, args.osiris_m, rank, flush, world)

    # --- slab geometry: the blowout workload with sheet plasma and sheet bunches ---
    slab = slab_leg(wake, torch, args.slab_steps, rank, flush, world) if args.slab_steps > 0 else None

    # --- the latency-bound case: one march of the linear workload, microseconds ---
    latency = latency_leg(wake, torch, stream) if args.latency else None

    # --- the ALU peaks of this GPU, measured now (the roofline's denominator) ---
    fma = fma_peak_leg(local)

    # --- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(cfg)
        pool.round()  # untimed: the workers' first step
        n = 2
        wall = sum(pool.round() for _ in range(n))
        pool.close()
        sps = oracle_step_rate(cfg, 2)
        cpu = {"value": plasma_pushes_per_step(cfg) * pool.procs * n / wall, "unit": "pushes/s",
               "cores": pool.procs, "kind": "oracle",
               "sample": f"{n} rounds of one beam step of the workload on each of {pool.procs} processes (one "
                         f"independent copy per core), after one untimed round; FP64 oracle",
               "one_thread": {"value": plasma_pushes_per_step(cfg) / sps, "unit": "pushes/s",
                              "sample": "2 beam steps of the workload, one host thread"}}

    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    alive = diag[0] + diag[3]
    flops_run = nbs * (march_flops(cfg) + alive * FLOP_PER_BEAM_PUSH)
    kern_s = sum(kern_ms) / len(kern_ms) / 1e3
    achieved = flops_run / kern_s / 1e12
    peak = fma["fp32_tflops"]
    default_workload = (cfg.nr, cfg.nxi, cfg.n_beam, nbs) == (512, 2048, 1 << 20, BEAM_STEPS)
    traffic = STEP_TRAFFIC_BYTES if default_workload and step_sources_hash() == STEP_TRAFFIC_SOURCES else None
    roof = {"kernel": "step_kernel<PolMixed>", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "peak_source": "measured: FP32 FMA micro-benchmark (paper_1411_3246_gb300/peak) in this run, "
                           f"median SM clock {fma['clocks']['sm_mhz']} MHz; nominal at {sm_mhz:.0f} MHz "
                           f"({src} peaks file's max clock): {fp32_peak_tflops(sm_mhz):.1f} TFLOP/s",
            "kernel_ms": 1e3 * kern_s, "kernel_share_of_run": kern_s * 1e3 / (sum(run_ms) / len(run_ms))}
    if rank == 0:
        line = {"metric": "plasma_pushes_per_s", "value": value, "unit": "pushes/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_dict(cfg, world, nbs),
                "beam_pushes_per_s": world * cfg.n_beam * nbs * args.steps / tot_s,
                "fp64_gpu": fp64, "mixed64": mixed64,
                "e2e": {"value": world * pushes * e2e_steps / e2e_s, "unit": "pushes/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 5 * 8},
                "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "batched": batched, "adjoint": adjoint,
                "large": large, "large_fp64": large_fp64, "facet": facet, "osiris": osiris, "slab": slab, "latency": latency, "alu_peaks": fma,
                "host_cores": {"nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))},
                "gpu_launches": KERNELS_PER_RUN * args.steps,
                "witness": {"mean_gamma": diag[1], "rms_gamma": diag[2], "alive": diag[0]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
