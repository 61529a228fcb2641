"""The multi-replica bench path on the host: two gloo ranks on the CPU (the layer has no
exchange step, so N GPUs run N independent replicas; only the timing is combined)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, v = bench.replica_throughput(100.0 + 50.0 * rank, K=10, world=world, dist=dist, device="cpu")
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in out:
        assert t == 150.0                      # max over ranks
        assert abs(v - 2 * 10 / 0.150) < 1e-9  # both replicas' layers over the slowest time


def test_single_replica_is_plain_throughput():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.replica_throughput(200.0, K=4, world=1)
    assert t == 200.0 and abs(v - 20.0) < 1e-12
