"""The multi-GPU form is replicas only (independent simulations per rank, no exchange): the
benchmark's rank logic - distinct replica seeds, the job time as the slowest rank's, the
aggregate value - checked with world_size 2 over gloo on the CPU."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import synth
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    cfg = synth.config_blowout(n_beam=64, nr=16, nxi=32)
    seed = bench.replica_seed(cfg.seed, r)
    t = bench.barrier_max(0.5 + r, w)  # rank r "took" 0.5 + r seconds
    bench.barrier(w)
    cfg.seed = seed
    out[r] = (seed, t, float(synth.beam_normals(cfg)[0, 0]))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replicas_world_size_two_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    seeds = [out[r][0] for r in range(world)]
    assert len(set(seeds)) == world  # independent replicas
    assert all(out[r][1] == 1.5 for r in range(world))  # every rank sees the slowest rank's time
    assert out[0][2] != out[1][2]  # different synthetic inputs
