"""Multi-rank path of bench.py on CPU: world size 2 over gloo (no GPU).

The solver shards only as independent replicas; the one collective is the max-reduction of
the step time.  Each rank reports a different time; both must see the slowest one and the
whole-job throughput of both replicas.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_replicas(100.0 + 50.0 * rank, 16, device="cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_max_time_and_sum_units():
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
    for rank, ms, value in res:
        assert ms == 150.0
        assert abs(value - 2 * 16 / 0.150) < 1e-9


def test_single_process_is_identity():
    import bench
    ms, value = bench.aggregate_replicas(200.0, 16)
    assert ms == 200.0 and abs(value - 80.0) < 1e-12
