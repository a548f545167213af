"""The multi-rank host logic of bench.py on the CPU: two gloo ranks (no GPU).
N > 1 runs independent replicas (no data-path collective): the only exchange is
the max-over-ranks timing reduction, and the reported value is the units all
ranks processed over the slowest rank's time.  The reference arm runs on rank 0
alone; the other ranks exit without work."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = [3.0, 5.0][rank]                  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, world, torch.device("cpu"))
        value = bench.aggregate_rate(2.0e9, world, ms_max)
        # replicas: the same shape of work per rank, different synthetic draws
        import workloads as wl
        w = wl.c1(n=256, seed=rank)
        q.put((rank, ms_max, value, w.X.shape, float(w.X[0, 0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ms_max, value, shape, x00 in res:
        assert ms_max == 5.0                                     # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 2.0e9 / 5e-3 / 1e9)    # both ranks' units over it
    assert res[0][3] == res[1][3] and res[0][4] != res[1][4]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""
