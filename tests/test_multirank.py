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


def _dying_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    bench.init_ranks("gloo", timeout_s=20.0)
    if rank == 1:
        os._exit(3)  # dies between steps, before the aggregation collective
    import time
    t0 = time.monotonic()
    try:
        bench.job_rate(100.0, 1e6, world, "cpu")
        q.put((rank, "no error", time.monotonic() - t0))
    except Exception as e:  # the survivor learns of the dead rank at its next collective
        q.put((rank, type(e).__name__, time.monotonic() - t0))


def test_dead_rank_surfaces_as_an_error_not_a_hang():
    """A rank that exits after joining: the other rank's next collective (the
    bench's max-over-ranks aggregation) raises within the process-group
    timeout instead of waiting forever."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        rank, outcome, waited = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert rank == 0 and outcome != "no error", outcome
    assert waited < 60.0
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
