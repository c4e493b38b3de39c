"""Multi-rank host logic of the replica runs (CPU, gloo, world size 2).

The MSFV path does not shard: each GPU solves its own instance.  These tests run the
same helpers bench.py uses on two CPU processes over gloo: distinct seeds per rank, the
barrier, MAX-over-ranks timing and the whole-job rate.  No GPU is touched.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1707_07598_gb300 import replicas as R  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R.barrier()
        # rank r pretends its timed region took 1 + r seconds
        slowest = R.max_over_ranks(1.0 + rank)
        rate = R.whole_job_rate(world, 5, slowest)
        seeds = R.replica_seeds(rank)
        out.put((rank, slowest, rate, seeds.model, seeds.truth, seeds.noise))
    finally:
        dist.destroy_process_group()


def test_rank_env_defaults_and_values():
    assert R.rank_env({}) == R.RankEnv(0, 1, 0)
    e = R.rank_env({"RANK": "3", "WORLD_SIZE": "4", "LOCAL_RANK": "1"})
    assert (e.rank, e.world, e.local) == (3, 4, 1)


def test_whole_job_rate():
    assert R.whole_job_rate(1, 10, 2.0) == 5.0
    assert R.whole_job_rate(4, 10, 2.0) == 20.0
    with pytest.raises(ValueError):
        R.whole_job_rate(0, 1, 1.0)
    with pytest.raises(ValueError):
        R.whole_job_rate(1, 1, 0.0)


def test_single_rank_max_is_identity():
    assert R.max_over_ranks(3.5) == 3.5
    R.barrier()  # no process group: a no-op


def test_two_rank_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time, and the job rate counts both ranks' units
    assert [r[1] for r in res] == [2.0, 2.0]
    assert [r[2] for r in res] == [5.0, 5.0]
    # replicas solve different problems
    assert len({r[3] for r in res}) == 2 and len({r[4] for r in res}) == 2
    assert len({r[5] for r in res}) == 2


def test_reference_arm_under_torchrun_rank1_exits_without_work(tmp_path):
    """bench.py --impl reference under a 2-rank launch: only rank 0 prints a line."""
    port = _free_port()
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
