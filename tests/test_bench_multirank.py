"""The multi-GPU path of bench.py on the CPU: two gloo ranks on 127.0.0.1.

Problems shard by rank with no data exchange (each rank draws its own seeded
batch), and the job time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = bench.workload_problems(6, rank_offset=rank)
    t = bench.max_over_ranks(0.5 + rank, dist)
    out[rank] = (float(np.sum([p.spot.sum() for p in probs])), t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    (s0, t0), (s1, t1) = out[0], out[1]
    assert s0 != s1                      # each rank prices its own problems
    assert t0 == t1 == 1.5               # both see the slowest rank's time
