"""The N > 1 path on CPU: replicas that only meet in the max-over-ranks
timing (gloo, world size 2), shards of the hard-leaf sum computed on CPU ranks
from their own starting values and added exactly, and the reference arm under
torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica does the same work (here: the oracle on a small x) in its own time
        local_ms = 100.0 + 50.0 * rank
        units = 10 ** 6
        value = oracle.pi_sieve(units)
        slowest = bench.max_over_ranks(local_ms, world)
        thr = bench.job_throughput(units, world, slowest / 1000.0)
        # shard partial sums are 128-bit integers: their sum over ranks must be exact
        total = bench.sum_over_ranks((rank + 1) * (1 << 100) - rank, world)
        q.put((rank, slowest, thr, value, total))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slowest, thr, value, total in res:
        assert slowest == 150.0                       # every rank sees the slowest replica's time
        assert thr == pytest.approx(2 * 10 ** 6 / 0.150)
        assert value == 78498                          # pi(10^6), Table 1
        assert total == 3 * (1 << 100) - 1
    assert res[0][1:] == res[1][1:]


def _shard_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r takes the r-th of `world` equal runs of 32 KiB sieve segments (983040
        # integers each) of [0, z], as pc_s2_hard_shard splits them, sieves only its range
        # and starts its carries from phi(L - 1, b) (Section 4); the ranks meet only to add
        # their 128-bit partial sums
        x, y, c = 10 ** 11, 2 * oracle.iroot3(10 ** 11), 5
        span = 983040
        nseg = (x // y) // span + 1
        s0, s1 = nseg * rank // world, nseg * (rank + 1) // world
        part, n = oracle.s2_hard_range(x, y, c, max(1, s0 * span), s1 * span)
        total = bench.sum_over_ranks(part, world)
        q.put((rank, total, n))
    finally:
        dist.destroy_process_group()


def test_shards_on_cpu_ranks_gloo():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    x, y, c = 10 ** 11, 2 * oracle.iroot3(10 ** 11), 5
    whole = oracle.leaf_sums(x, y, c)
    assert res[0][1] == res[1][1] == whole["S2_hard"]
    assert res[0][2] + res[1][2] == whole["n_hard"]
    assert res[0][2] > 0 and res[1][2] > 0


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2
