"""The N > 1 path on CPU: two gloo ranks combine their timings the way
bench.py does under torchrun (slowest rank's time, all ranks' attempts)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2604_08250_gb300 import replicas
        value, t = replicas.job_throughput(times[rank], 1e9, dist)
        dist.barrier()
        out.put((rank, value, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_slowest_time_and_all_attempts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [250.0, 400.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 400.0
        assert value == pytest.approx(2 * 1e9 / 0.4)


def test_single_process_without_group():
    from paper_2604_08250_gb300 import replicas
    value, t = replicas.job_throughput(500.0, 1e9)
    assert t == 500.0 and value == pytest.approx(2e9)
    with pytest.raises(ValueError):
        replicas.job_throughput(0.0, 1.0)
