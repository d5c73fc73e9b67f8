"""The multi-GPU shape of the benchmark is replicas only (no data-path
collective): each rank runs the whole path on its own problem, and the job's
time is the slowest rank's.  These CPU tests run two ranks over gloo and check
that host logic: the max over ranks, the whole-job value, and that the
reference arm does its work on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        ms = bench.slowest_ms(10.0 + 5.0 * rank, dist)  # rank 1 is the slow one
        q.put((r, w, local, ms, bench.job_value(w, 1.0e15, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, ms, value in out:
        assert w == 2 and local == r
        assert ms == 15.0
        assert value == pytest.approx(2 * 1.0e15 / 15.0e-3 / 1e12)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.slowest_ms(12.5) == 12.5
    assert bench.job_value(1, 2.0e12, 1000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_sample", lambda *a, **k: called.append(1))
    args = types.SimpleNamespace(config="c3", ref_rows=64, warmup=0, steps=1)
    assert bench.run_reference(args) == 0
    assert not called
