"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks.

Each rank advances its own cavity (replicas only); the job's time is the
maximum over ranks and its throughput the units of all ranks over that
time; only rank 0 prints, and the reference arm runs on rank 0 alone.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    times = bench.max_over_ranks([1.0 + r, 10.0 - 3 * r], w, "cpu")
    q.put((r, w, local, times, bench.job_value(100, w, times[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_to_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, times, value) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert times == [2.0, 10.0]          # max over ranks, per entry
        assert value == pytest.approx(100.0)  # 100 units x 2 ranks / 2.0 s


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks([3.5, 1.25], 1, "cpu") == [3.5, 1.25]
    assert bench.job_value(10, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
