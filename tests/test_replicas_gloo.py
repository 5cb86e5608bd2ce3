"""Host logic of the multi-replica bench on CPU: two gloo ranks that each ran the same number
of steps in different times report the slowest rank's time and every rank's steps; under a
distributed launch the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]                 # the second rank is slower
    value, tmax = bench.replica_throughput(elapsed, 5, world, dist, "cpu")
    q.put((rank, value, tmax, bench.dist_env()[:2]))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, env in out:
        assert tmax == pytest.approx(3.0)                 # the slowest rank bounds the job
        assert value == pytest.approx(2 * 5 / 3.0)        # every rank's steps count
        assert env == (rank, 2)


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(2.0, 4, 1) == (2.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())          # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
