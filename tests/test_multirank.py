"""Multi-rank aggregation of bench.py (weak scaling, one realization per rank),
exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, slowest = bench.job_rate(100.0 + 50.0 * rank, 1e6 * (rank + 1), world, "cpu")
    q.put((rank, value, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_total_work_over_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in res:
        assert slowest == 150.0
        assert abs(value - 3e6 / 0.150) < 1e-6 * value


def test_job_rate_single_rank():
    import bench
    value, t = bench.job_rate(50.0, 1e6, 1, "cpu")
    assert t == 50.0 and abs(value - 2e7) < 1e-3
