"""Replica bench logic across ranks (gloo, world size 2, CPU): the job's time
is the slowest rank's and the rate counts every rank's solves. The solver
itself does not shard (independent solves, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t_max = bench.reduce_max(t_local)
    value = bench.replica_throughput(dist.get_world_size(), 4, t_max)
    q.put((rank, t_max, value, bench.dist_setup(world)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value, (r, w, l) in out:
        assert t_max == 150.0
        assert value == pytest.approx(2 * 4 / 0.150)
        assert (r, w) == (rank, 2)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.replica_throughput(1, 5, 2000.0) == pytest.approx(2.5)
