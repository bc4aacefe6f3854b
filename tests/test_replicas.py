"""The multi-GPU form is replicas only: each rank steps its own independent solve
and the whole-job throughput is all ranks' steps over the slowest rank's time.
Checked here with two gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
        value, total_ms = bench.replica_throughput(local_ms, steps=10)
        out.put((rank, value, total_ms))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, total_ms in res:
        assert total_ms == pytest.approx(200.0)  # the slowest rank's time
        assert value == pytest.approx(world * 10 / 0.2)  # all ranks' steps / that time


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    value, total_ms = bench.replica_throughput(250.0, steps=5)
    assert total_ms == 250.0 and value == pytest.approx(20.0)
