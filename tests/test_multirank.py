"""The multi-GPU path is replicas only: every rank runs an independent
registration workload and the job's throughput is (ranks x units per rank) /
(slowest rank's time).  The host-side aggregation runs here with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as td

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
        ms = bench.max_over_ranks(local_ms)
        value = bench.replica_throughput(20, world, ms)
        q.put((rank, ms, value))
    finally:
        td.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 150.0                       # max over ranks, seen by every rank
        assert abs(value - 2 * 20 / 0.150) < 1e-9


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(10, 1, 500.0) == 20.0
