"""The host-side logic of a multi-rank benchmark run, on CPU with two gloo ranks.

Tracking and fusion of one scene do not shard; `bench.py --gpus N` runs N independent replicas of
the workload, one per rank, with no data-path collective.  What spans the ranks is the timing:
every rank's timed interval is reduced to the largest (the slowest rank bounds the job), and the
job's throughput is N times one replica's units over that time.  The reference arm runs on rank 0
only; the other ranks exit at once without work.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_max = bench.reduce_max(times[rank], world, torch.device("cpu"))
    q.put((rank, t_max, bench.job_rate(world, 1000.0, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_bounds_the_job_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.25, 0.40]  # rank 1 is the slower replica
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, t_max, rate in got:
        assert t_max == 0.40  # every rank holds the maximum
        assert rate == pytest.approx(2 * 1000.0 / 0.40)  # N replicas' units over the slowest time


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.reduce_max(0.3, 1, None) == 0.3
    assert bench.job_rate(1, 600.0, 0.3) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
