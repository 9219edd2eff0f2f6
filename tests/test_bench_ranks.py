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


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the CPU oracle on the same workload and
    metric and prints one JSON line with the reference arm's keys."""
    import json
    import subprocess
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["metric"] == "condense+Cholesky ms/IPM iter" and d["unit"] == "ms/iter"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
