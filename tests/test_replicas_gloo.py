"""The multi-GPU form of the benchmark is N independent replicas (the path does not shard): the
slowest rank's time is taken with an all-reduce MAX and the whole-job rate counts every rank's
levels.  These tests run that reduction over two gloo ranks on CPU, and check that the reference
arm's other ranks exit without work."""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 180.0][rank]  # rank 1 is the slow replica
    ms_max = bench.max_over_ranks(ms, world)
    rate = bench.replica_rate(10 * 8, ms_max / 1e3, world)  # 10 steps of 8 levels per rank
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms_max, rate))


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 180.0  # every rank sees the slowest replica's time
        assert rate == pytest.approx(2 * 80 / 0.180)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.replica_rate(80, 0.5, 1) == 160.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
