"""The multi-process side of bench.py on CPU (gloo, world size 2): replicas
get disjoint global bitstring indices and the timing reduction takes the
slowest rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    worst, value = bench.aggregate_timing(local_ms, world, 10_000, 4, dist)
    seed, base = bench.replica_plan(rank, world, 10_000)
    dist.barrier()
    q.put((rank, worst, value, seed, base))
    dist.destroy_process_group()


def test_replicas_and_timing_reduction_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, v0, s0, b0), (r1, w1, v1, s1, b1) = res
    assert w0 == w1 == 150.0  # the slowest rank's time on every rank
    assert v0 == v1 == 2 * 10_000 * 4 / 0.150
    assert s0 != s1 and (b0, b1) == (0, 10_000)
