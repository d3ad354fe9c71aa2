"""Multi-rank host logic of the benchmark (replicas, no data-path collective),
run as two gloo ranks on the CPU: the job time is the slowest rank's and the
throughput counts every rank's nodes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, mlups = bench.replica_throughput(100.0 * (rank + 1), 1_000_000, 10)
    q.put((rank, ms, mlups))
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, mlups in res:
        assert ms == pytest.approx(200.0)                  # the slower rank sets the job time
        assert mlups == pytest.approx(2 * 1e6 * 10 / 0.2 / 1e6)  # both ranks' node updates


def test_single_process_is_identity():
    import bench
    ms, mlups = bench.replica_throughput(50.0, 1000, 100)
    assert ms == 50.0 and mlups == pytest.approx(1000 * 100 / 0.05 / 1e6)
