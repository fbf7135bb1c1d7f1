"""The multi-GPU bookkeeping of bench.py on two gloo ranks (CPU): each rank runs its own
replica, the elapsed time is the maximum over ranks and the whole-job rate counts every
rank's work; the reference arm's ranks other than 0 do nothing."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(1000, 4, world, ms / 1e3)
    dist.barrier()
    out.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, ms, rate in res:
        assert ms == 15.0
        assert abs(rate - 1000 * 4 * 2 / 0.015 / 1e6) < 1e-12


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert abs(bench.whole_job_rate(4194304, 20, 1, 0.3) - 4194304 * 20 / 0.3 / 1e6) < 1e-9
