"""bench.py's multi-rank host logic on CPU ranks (gloo, world size 2).

Each rank solves its own seeded system with no collective on the data path;
the only exchange is the max over ranks of the timed region, and the job
throughput counts every rank's solves within that max time.
"""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.rank_env()
        # rank-dependent "timed region" lengths: the job time is the slowest rank's
        t_ms = 1000.0 * (rank + 1)
        dist.barrier()
        t_max = bench.max_over_ranks(t_ms, w, "cpu")
        dist.barrier()
        q.put((r, w, local, bench.system_seed(r), t_max, bench.job_throughput(3, w, t_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_is_max_and_throughput_counts_all_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    # independent systems per rank
    assert out[0][3] != out[1][3]
    # every rank sees the slowest rank's time; 3 solves per rank in 2 s
    assert all(o[4] == 2000.0 for o in out)
    assert all(o[5] == pytest.approx(3.0) for o in out)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(2, 1, 500.0) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload = bench.DEFAULT_WORKLOAD
        warmup, steps = 3, 1
    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
