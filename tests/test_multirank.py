"""The N>1 bench path: each rank is one GPU running the whole workload as an
independent replica (no collective on the data path); the job's time is the
slowest rank's, its work the sum over ranks, and only rank 0 reports.
Checked with world_size-2 gloo process groups on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: slowest time 1.5 + r, counters that differ by rank
        t, sums = bench.reduce_over_ranks(dist, "cpu", 1.5 + rank, [1000 * (rank + 1), rank, 7])
        q.put((rank, t, sums))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
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
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, sums in got:
        assert t == 2.5                         # max over ranks
        assert sums == [3000.0, 1.0, 14.0]      # sum over ranks


def test_reduce_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 3.25, [5, 6]) == (3.25, [5.0, 6.0])


def test_reference_arm_under_torchrun_world2_rank0_reports_alone():
    """`bench.py --impl reference` launched by torchrun on two ranks: rank 0
    prints the one JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    env = dict(os.environ)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--workload", "planted1e4+grid64"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
