"""The N > 1 path of bench.py on CPU: two gloo ranks.

The path shards by problem (independent problems, no exchange on the data
path); the only collective is the max over ranks of the timed duration.  These
tests run that host logic with world_size 2 over gloo on 127.0.0.1, and the
reference arm under a real two-process launch, where rank 1 must exit without
work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.shard_seeds(rank)
        mx = bench.reduce_max(10.0 + rank, world)
        total = bench.reduce_sum(1.0 + rank, world)
        out.put((rank, seeds, mx, total))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_disjoint_problems_and_agree_on_the_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, free_port_cached(), q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    s0, s1 = set(res[0][1]), set(res[1][1])
    assert len(s0) == len(s1) == 256 and not (s0 & s1)
    assert min(s0) == 4000 and min(s1) == 4256
    assert res[0][2] == res[1][2] == 11.0
    # certified solves are summed over ranks (the whole-job value)
    assert res[0][3] == res[1][3] == 3.0


_PORT = None


def free_port_cached():
    global _PORT
    if _PORT is None:
        _PORT = free_port()
    return _PORT


@pytest.mark.slow
def test_reference_arm_under_two_process_launch():
    """bench.py --impl reference under torchrun with 2 ranks: rank 0 prints one
    JSON line for the oracle, rank 1 exits 0 without work."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
