"""Replica coordination on CPU (gloo, two ranks): the timing reduction the
multi-GPU bench uses, the whole-job rate, and the sharding of independent
systems. No data crosses ranks on the solve path; only timings are reduced."""
import os
import socket
import subprocess
import sys

import pytest

from paper_2505_09727_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    replicas.init("gloo")
    replicas.barrier()
    # rank-dependent step times: the job time is the slowest rank's
    got = replicas.max_over_ranks([1.0 + rank, 10.0 * (world - rank)])
    rate = replicas.whole_job_rate(1000, world, got[0])
    out.put((rank, got, rate, list(replicas.shard(10, rank, world))))
    replicas.finalize()


def test_two_rank_timing_reduction_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate, share in res:
        assert got == [2.0, 20.0]                 # max over both ranks, on every rank
        assert rate == pytest.approx(1000 * 2 / 2.0)
    assert res[0][3] + res[1][3] == list(range(10))


@pytest.mark.parametrize("n,world", [(10, 3), (64, 8), (5, 8), (0, 2)])
def test_shard_is_a_partition(n, world):
    parts = [list(replicas.shard(n, r, world)) for r in range(world)]
    flat = [i for p in parts for i in p]
    assert flat == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_single_process_is_identity():
    assert replicas.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
