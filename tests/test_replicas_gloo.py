"""The multi-GPU path of the benchmark runs independent replicas (one per
rank, no collective on the data path); the ranks only agree on the slowest
replica's time.  That reduction runs here as two gloo processes on the CPU."""
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


def _worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, ws)   # rank 1 is the slow replica
    same = bench.max_over_ranks(3.25, ws)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, same))


def test_slowest_replica_time_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 15.0, 3.25), (1, 15.0, 3.25)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
