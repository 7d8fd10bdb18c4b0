"""The benchmark's multi-rank path on the CPU: two gloo ranks (127.0.0.1)
combine their timings the way bench.py does -- element-wise maximum over the
ranks, and the whole-job rate as all ranks' units per second of the slowest
rank (independent replicas, weak scaling) -- and the reference arm leaves
every rank but 0 without work."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 10.0 - 3 * rank]            # rank 1 slower on the first
        got = bench.max_over_ranks(dist, mine, "cpu")
        q.put((rank, got, bench.whole_job_rate(world, 1000, got[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [2.0, 10.0]                        # max over ranks, per entry
        assert rate == pytest.approx(2 * 1000 / 2.0)     # all units / slowest rank's time


def test_single_process_values_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 500, 2.0) == 250.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""
