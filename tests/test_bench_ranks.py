"""The multi-rank (replica) path of bench.py, on CPU with two gloo ranks: the
job's time is the slowest rank's timed region, its rate counts every rank's
cells, and the reference arm does its work on rank 0 alone."""
import argparse
import io
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import os

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # each rank times a different region: 10 ms on rank 0, 20 ms on rank 1
    t = bench.job_time_ms(10.0 * (rank + 1), ws, "cpu")
    q.put((rank, t, bench.job_rate(ws, 1000, 4, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_the_rate_counts_every_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    ws, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in got:
        assert t == 20.0
        # 2 ranks x 1000 cells x 4 steps over the slowest rank's 20 ms
        assert rate == pytest.approx(2 * 1000 * 4 / 0.020)


def test_single_rank_time_is_its_own():
    import bench
    assert bench.job_time_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 256 ** 3, 10, 250.0) == pytest.approx(256 ** 3 * 10 / 0.25)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=1, warmup=3, cpu_sample_nodes=10)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) is None
    assert out.getvalue() == ""
