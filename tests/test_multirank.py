"""The N > 1 path of bench.py: each rank runs its own lattice (replicas only,
no data-path collective); the job rate divides the total work by the slowest
rank's time.  Checked with two gloo ranks on CPU."""
import os
import socket
import sys
from pathlib import Path

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parent.parent


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, str(ROOT))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_local = [2.0, 3.0][rank]  # rank 1 is the slowest
    value, t = bench.aggregate(dist, world, sites_per_step=1000, steps=50, t_local=t_local)
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_use_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in out:
        assert t == 3.0
        assert value == pytest.approx(2 * 1000 * 50 / (3.0 * 1e9))


def test_single_rank_needs_no_collective():
    sys.path.insert(0, str(ROOT))
    import bench

    value, t = bench.aggregate(None, 1, 4096 * 4096, 10, 0.5)
    assert t == 0.5 and value == pytest.approx(4096 * 4096 * 10 / 0.5e9)
