"""The multi-process path of bench.py, on CPU with the gloo backend (world size 2).

The method has no exchange step between independent runs, so bench.py runs
one replica per GPU. Each rank reports its own time, the slowest rank sets
the whole job's time (max over ranks), and rank 0 alone prints. These tests
cover that host logic without a GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        local_ms = 10.0 + 5.0 * rank                       # rank 1 is the slower replica
        worst = bench.reduce_max(local_ms, world, "cpu")
        value = bench.whole_job_value(1024, 10, 100, world, worst / 1e3)
        q.put((rank, w, r, loc, worst, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, loc, worst, value in out:
        assert (w, r, loc) == (2, rank, rank)
        assert worst == 15.0                                # both ranks see the slowest time
        assert value == pytest.approx(2 * 1024 * 10 * 100 / 0.015)


def test_reference_arm_prints_on_rank0_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 3, 3
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_single_process_defaults(monkeypatch):
    import bench
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_max(3.5, 1, "cpu") == 3.5
