"""Multi-rank plumbing of bench.py on the CPU (gloo, world size 2).

The method is not sharded across GPUs: under torchrun every rank runs an
independent replica, and the only cross-rank operations are the barrier, the
maximum of the ranks' timed durations and the sum of the cells they processed
(the reported throughput is all cells / slowest rank).  No data-path
collective exists.  This test runs those helpers in two gloo processes."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    dist.init_process_group(backend="gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    ms = 10.0 + 5.0 * rank                   # each replica's timed duration
    cells = 1000.0 * (rank + 1)              # cells x steps each replica processed
    tmax = bench.reduce_max(dist, ms)
    csum = bench.reduce_sum(dist, cells)
    q.put((rank, tmax, csum))
    dist.destroy_process_group()


def test_replica_reductions_over_two_gloo_ranks():
    import multiprocessing as mp
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
    for rank, tmax, csum in out:
        assert tmax == pytest.approx(15.0)     # slowest replica
        assert csum == pytest.approx(3000.0)   # cells of all replicas
