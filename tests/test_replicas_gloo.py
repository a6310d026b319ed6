"""The multi-GPU path is replicas only (one array per rank, no collective on the data path):
what crosses ranks is the benchmark's timing -- the slowest rank's time, seen by every rank,
and the whole-job throughput computed from it.  Checked with world size 2 over gloo on CPU, plus
the reference arm's rank rule (rank 0 alone runs it)."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from conftest import ROOT


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [12.5, 20.0]
    got = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
    value = bench.replica_throughput(world, 1000, 4, got)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, value))


def test_max_over_ranks_world_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    # 2 replicas x 4 steps x 1000 keys in 20 ms
    assert all(abs(r[2] - 2 * 4 * 1000 / 0.020 / 1e9) < 1e-12 for r in res)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
