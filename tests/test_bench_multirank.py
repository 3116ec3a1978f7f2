"""Host logic of the multi-GPU (replicas) layout of bench.py, run as two
gloo ranks on the CPU: the step time is the maximum over ranks and the
value counts every rank's unknowns."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms_list, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate(ms_list[rank], 1000, world, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms_list = [2.0, 5.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms_list, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 5.0
        assert value == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate(4.0, 500, 1) == (4.0, 500 / 4e-3)
