"""The multi-rank path of bench.py (replicas: no data-path collective, the
slowest rank's time, whole-job throughput) on CPU with gloo, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    worst = bench.max_over_ranks(ms, world, torch.device("cpu"))
    rate = bench.job_rate(16, 10, world, worst)
    q.put((rank, worst, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for _, worst, rate in res:
        assert worst == 150.0                       # max over ranks
        assert rate == pytest.approx(2 * 16 * 10 / 0.150)   # all ranks' views / slowest time
