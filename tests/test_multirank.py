"""Host logic of the multi-GPU (replica) path on CPU with 2 gloo ranks: the bench's
aggregation takes the slowest rank's time and counts every rank's work."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 3.0][rank]
    value, t = bench.aggregate(dist, elapsed, 60.0)
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
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
    for rank, value, t in out:
        assert t == 3.0                       # max over ranks
        assert abs(value - 2 * 60.0 / 3.0) < 1e-12


def test_single_process_aggregation():
    import bench
    value, t = bench.aggregate(None, 0.5, 10.0)
    assert t == 0.5 and value == 20.0
