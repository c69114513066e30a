"""The N > 1 path of bench.py is replicas only: every rank solves its own copy
of the workload and the ranks exchange one scalar, the slowest rank's time.
Two gloo ranks on the CPU check that exchange and the whole-job value."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    got = bench.max_over_ranks(ms, torch.device("cpu"))
    q.put((rank, got, bench.whole_job_value(64, 3, world, got)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == 150.0
        # 2 ranks x 3 steps x 64 units in 150 ms
        assert value == pytest.approx(2 * 3 * 64 / 0.150)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
