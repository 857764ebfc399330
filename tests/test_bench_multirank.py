"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the timed
region's time is the maximum over ranks, the job value counts every rank's
iterations, and the reference arm runs on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench._max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
    value = bench._job_value(200, ws, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value))


def test_max_over_ranks_and_job_value_gloo():
    pytest.importorskip("torch")
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, ms, value in out:
        assert ms == 15.0  # the slower rank's time on every rank
        assert value == pytest.approx(200 * 2 / 0.015)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_value(100, 1, 50.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="small_40cube", steps=1, warmup=3)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
