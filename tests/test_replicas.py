"""Multi-GPU runs are replicas (one independent tree per rank, no data exchange). The cross-rank
host logic of a timed run — barrier, the slowest rank's time, the whole-job rate — checked with
two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1610_00823_gb300 import replicas
        replicas.barrier(dist)
        slowest = replicas.max_over_ranks(1.5 + rank, dist)  # rank times 1.5 ms and 2.5 ms
        q.put((rank, slowest, replicas.whole_job_rate(1000, slowest, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 2.5
        assert rate == pytest.approx(2 * 1000 / 2.5e-3)


def test_single_process_needs_no_group():
    from paper_1610_00823_gb300 import replicas
    replicas.barrier(None)
    assert replicas.max_over_ranks(3.0, None) == 3.0
    assert replicas.whole_job_rate(10, 2.0, 1) == pytest.approx(5000.0)
