"""Multi-process (replica) logic of bench.py on CPU with the gloo backend:
each rank runs an independent replica with its own seed and Philox stream,
and the job's figures are the slowest rank's time and the sum of the node
updates. The path itself has no data exchange between ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    p = bench.workload_params(rank)
    # rank r times (10 + r) ms for (1000 * (r + 1)) node updates
    ms, nodes = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, (p["seed"], p["sim_id"]))
    if rank == 0:
        out.put((ms, nodes, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_and_seeds_world_size_2():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    ms, nodes, seeds = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ms == 11.0          # the slowest rank
    assert nodes == 3000.0     # all ranks' work
    assert len(set(seeds)) == world  # independent replicas


PORT = _free_port()
