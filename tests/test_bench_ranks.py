"""The multi-GPU form of bench.py is replicas only: every rank runs its own
copy of the workload, and the ranks exchange nothing but the timing.  This
checks that reduction with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    total, launches = bench.reduce_over_ranks(10.0 * (rank + 1), 2 + rank, "cpu")
    q.put((rank, total, launches))
    dist.destroy_process_group()


def test_replicas_reduce_max_time_and_sum_launches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, launches in got:
        assert total == 20.0      # the slowest rank's time
        assert launches == 5      # 2 + 3 kernels
