"""Benchmark: plasma pushes/s of the quasi-static wake step on the blowout two-bunch workload.

Workload (one "step" = one beam time step: beam deposit -> xi-march -> beam push): warm
plasma u_th = 0.01, Nr = 512 over 8 k_p^-1, Nxi = 2048 over 12 k_p^-1, 8 rings per cell
(4096 rings per slice), two-bunch Eq. 12 driver n_b/n_p = 8, sigma_r = 0.2, sigma_z = 0.6,
gamma = 4e4, witness 4.5 behind with 30% of the drive charge, 1,048,576 beam macroparticles,
dt = 5.  One step = 4096 x 2048 = 8,388,608 plasma pushes and 1,048,576 beam pushes.

Arms:
  default           the library's mixed-precision form (FP32 rings and fields, wide sums)
  --impl reference  the FP64 CPU oracle on the host cores (bounded sample of the same steps)

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream; between timed steps a 512 MB buffer is written to flush L2.  The JSON
line also carries the plain-FP64 GPU path (same scheme, FP64 throughout), an end-to-end
number through the C ABI from pinned host buffers, the march kernel's roofline and the
oracle CPU baseline.
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

# FP32 operations per plasma push of the mixed march (one ring advanced one slice: two
# field stages and two Cartesian moves; an FMA counts 2, a divide or sqrt 1), and the
# per-node work of the two stages amortised over the rings of the slice.  Counted from
# the kernel source, see the design doc.
FLOP_PER_PUSH = 236.0
FLOP_PER_NODE_STAGE = 62.0


def workload():
    return synth.config_blowout(n_beam=1 << 20)


def plasma_pushes_per_step(cfg):
    return cfg.nr * cfg.ppc * cfg.nxi


def march_flops(cfg):
    return plasma_pushes_per_step(cfg) * FLOP_PER_PUSH + 2 * cfg.nxi * (cfg.nr + 1) * FLOP_PER_NODE_STAGE


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


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
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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


def run_reference(args, world, rank):
    """--impl reference: the oracle on the host cores, same metric and workload."""
    if rank != 0:
        return
    cfg = workload()
    import oracle
    pl = oracle.plasma_init(cfg, synth.plasma_normals(cfg))
    bm = oracle.beam_init(cfg, synth.beam_normals(cfg))
    for _ in range(args.warmup):
        oracle.run(cfg, pl, bm, 1)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.run(cfg, pl, bm, 1)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    v = plasma_pushes_per_step(cfg) * args.steps / tot
    line = {"impl": "reference", "metric": "plasma_pushes_per_s", "value": v, "unit": "pushes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(cfg, world),
            "cpu_baseline": {"value": v, "unit": "pushes/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full beam steps of the workload, one host thread"},
            "e2e": {"value": v, "unit": "pushes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(cfg, world):
    return {"workload": "blowout two-bunch warm plasma, Nr=512 x Nxi=2048, 8 rings/cell, 1M beam particles, dt=5",
            "nr": cfg.nr, "nxi": cfg.nxi, "ppc": cfg.ppc, "n_beam": cfg.n_beam, "u_th": cfg.u_th,
            "plasma_pushes_per_step": plasma_pushes_per_step(cfg), "beam_pushes_per_step": cfg.n_beam,
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--march-only", type=int, default=0,
                    help="run this many mixed marches of the workload and exit (profiling)")
    ap.add_argument("--nr", type=int, default=0, help="override Nr (profiling a smaller case)")
    ap.add_argument("--nxi", type=int, default=0, help="override Nxi (profiling a smaller case)")
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
    cfg.seed += 1000 * rank  # independent replicas
    nm_p = torch.from_numpy(synth.plasma_normals(cfg)).pin_memory()
    nm_b = torch.from_numpy(synth.beam_normals(cfg)).pin_memory()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pushes = plasma_pushes_per_step(cfg)

    if args.march_only:
        sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
        with torch.cuda.stream(stream):
            wake.wake_load_plasma(sim.h, 0, nm_p.cuda(non_blocking=True))
            wake.wake_load_beam(sim.h, 0, nm_b.cuda(non_blocking=True))
            wake.wake_beam_deposit(sim.h)
            for _ in range(args.march_only):
                wake.wake_plasma_march(sim.h)
        stream.synchronize()
        st = sim.status(0)
        sim.close()
        print(json.dumps({"march_only": args.march_only, "nr": cfg.nr, "nxi": cfg.nxi, "status": st}))
        return

    def timed_steps(prec, k, w, march_events=True):
        sim = wake.Simulations([cfg], prec, stream)
        with torch.cuda.stream(stream):
            wake.wake_load_plasma(sim.h, 0, nm_p.cuda(non_blocking=True))
            wake.wake_load_beam(sim.h, 0, nm_b.cuda(non_blocking=True))
            for _ in range(w):
                wake.wake_step(sim.h, 1)
        stream.synchronize()
        step_ms, march_ms = [], []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev[0].record(stream)
                wake.wake_beam_deposit(sim.h)
                ev[1].record(stream)
                wake.wake_plasma_march(sim.h)
                ev[2].record(stream)
                wake.wake_beam_push(sim.h)
                ev[3].record(stream)
            stream.synchronize()
            step_ms.append(ev[0].elapsed_time(ev[3]))
            march_ms.append(ev[1].elapsed_time(ev[2]))
        st = sim.status(0)
        diag = sim.diagnostics()[0]
        sim.close()
        if st != wake.WAKE_OK:
            raise RuntimeError(f"simulation status {st}: {wake.wake_last_error()}")
        return step_ms, march_ms, diag

    # --- mixed-precision arm (the headline) ---
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, march_ms, diag = timed_steps(wake.WAKE_MIXED, args.steps, args.warmup)
        torch.cuda.synchronize()
    barrier(world)
    clocks = clk.summary()
    tot_s = barrier_max(sum(step_ms) / 1e3, world)
    value = world * pushes * args.steps / tot_s
    march_s = sum(march_ms) / 1e3 / args.steps

    # --- plain FP64 GPU path, same workload ---
    fp64 = None
    if args.fp64_steps > 0:
        s64, m64, _ = timed_steps(wake.WAKE_FP64, args.fp64_steps, 1)
        t64 = barrier_max(sum(s64) / 1e3, world)
        fp64 = {"value": world * pushes * args.fp64_steps / t64, "unit": "pushes/s",
                "ms_per_step": 1e3 * t64 / args.fp64_steps, "steps": args.fp64_steps}

    # --- end to end through the C ABI from pinned host buffers: a one-step run per step ---
    e2e_steps = max(1, min(args.steps, 5))
    h2d = nm_p.numel() * 8 + nm_b.numel() * 8
    diag_host = None
    e2e_ms = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = wake.Simulations([cfg], wake.WAKE_MIXED, stream)
        with torch.cuda.stream(stream):
            dp = nm_p.cuda(non_blocking=True)
            db = nm_b.cuda(non_blocking=True)
            wake.wake_load_plasma(sim.h, 0, dp)
            wake.wake_load_beam(sim.h, 0, db)
            wake.wake_step(sim.h, 1)
        diag_host = sim.diagnostics()  # synchronous device -> host read
        sim.close()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_s = barrier_max(sum(e2e_ms) / 1e3, world)

    # --- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = 8
        sps = oracle_step_rate(cfg, n)
        cpu = {"value": pushes / sps, "unit": "pushes/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} full beam steps of the workload (FP64 oracle, one host thread)"}

    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    achieved = march_flops(cfg) / march_s / 1e12
    peak = fp32_peak_tflops(sm_mhz)
    roof = {"kernel": "march_kernel<PolMixed>", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (max clock of {src} peaks file)",
            "march_ms": 1e3 * march_s}
    if rank == 0:
        line = {"metric": "plasma_pushes_per_s", "value": value, "unit": "pushes/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_dict(cfg, world),
                "beam_pushes_per_s": world * cfg.n_beam * args.steps / tot_s,
                "fp64_gpu": fp64,
                "e2e": {"value": world * pushes * e2e_steps / e2e_s, "unit": "pushes/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 5 * 8},
                "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": 4 * args.steps,
                "witness": {"mean_gamma": diag[1], "rms_gamma": diag[2], "alive": diag[0]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
