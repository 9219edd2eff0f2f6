"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the
instance shards cover every instance exactly once, and the aggregation takes
the slowest rank's time and the sum of the ranks' units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_shards_partition_the_instances():
    for world in (1, 2, 3, 4, 8):
        seen = sorted(i for r in range(world) for i in bench.shard(96, r, world))
        assert seen == list(range(96))
        sizes = [len(bench.shard(96, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        units = len(bench.shard(96, rank, world))
        t, n = bench.aggregate(1.0 + rank, units, dist, "cpu")
        out[rank] = (t, n)
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 96)


def test_aggregate_alone_is_identity():
    assert bench.aggregate(3.5, 7) == (3.5, 7)
