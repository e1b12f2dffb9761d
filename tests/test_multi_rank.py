"""The N>1 path of bench.py on CPU: independent replicas, max-over-ranks
timing, whole-job rate = all ranks' iterations / slowest rank's time
(world size 2, gloo)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    rate, total = bench.whole_job_rate(local_ms, 10, world, dist, torch.device("cpu"))
    q.put((rank, rate, total))
    dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
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
    for rank, rate, total in out:
        assert total == pytest.approx(250.0)
        assert rate == pytest.approx(2 * 10 / 0.25)


def test_single_rank_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rate, total = bench.whole_job_rate(200.0, 20, 1)
    assert rate == pytest.approx(100.0) and total == 200.0
