"""Multi-GPU = independent replicas: the rank logic of bench.py on CPU.

Two gloo processes stand in for two GPUs: the job's time is the slowest
rank's (max over ranks), every rank's units count toward the value, and only
rank 0 runs and prints the reference arm.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        got = bench.max_over_ranks(times[rank], dist, "cpu")
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_time_is_the_slowest_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [123.5, 456.25]
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 456.25, 1: 456.25}


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    args = SimpleNamespace(gpus=2, steps=1, warmup=0, workload="gmm5d_1m_f32",
                           linkages=["ward"], cpu_cap=5.0, ref_n=300)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args)
    assert out.getvalue() == ""  # other ranks exit without work
    monkeypatch.setenv("RANK", "0")
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args)
    line = json.loads(out.getvalue())
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["unit"] == "points/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
