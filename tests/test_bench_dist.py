"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): the job
time is the slowest rank's, the value counts every rank's replica, and the
reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.slowest_rank_ms(10.0 * (rank + 1), world)
    q.put((rank, ms, bench.job_value(1000, world, ms)))
    dist.destroy_process_group()


def test_slowest_rank_and_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 20.0                      # max over ranks
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_oracle_sampler_extrapolation():
    """The CPU baseline's sampler: every bin below the degree cap that has an
    affordable vertex is sampled, the per-row timers are positive where the
    oracle computed rows, the estimate covers the sampled bins' vertices, and
    the all-core throughput is at least the one-core one."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import graphgen as gg
    g = gg.rmat(12, 16, seed=2)
    s = bench.OracleSampler(g, per_bin=2, threads=2, seed=1)
    deg = np.diff(g.rowptr)
    assert s.nb_cap >= 1 << 12
    for b, cand in s.cands.items():
        assert (np.floor(np.log2(np.maximum(deg[cand], 1))).astype(int)[deg[cand] > 0] == b).all()
        assert (deg[cand] < s.deg_cap).all()
    wall, est = s.step()
    assert wall > 0 and est > 0
    v_all, v_one = s.values(est)
    assert v_all >= v_one > 0
    assert "thread-seconds" in s.describe(1, est)
