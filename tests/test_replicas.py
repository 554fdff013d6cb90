"""Host logic of the multi-GPU form (independent replicas, weak scaling) on
CPU with two gloo ranks: the timed region is the slowest rank's, the value
counts every rank's units, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(times[rank], world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world = 2
    times = [12.5, 30.25]
    out = mp.get_context("spawn").Manager().dict()  # no fork of a threaded process
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    assert out[0] == out[1] == max(times)


def test_aggregate_rate_counts_every_rank():
    # 2 replicas x 1e6 units x 5 steps in 100 ms (the slowest rank's time)
    assert bench.aggregate_rate(2, 10**6, 5, 100.0) == pytest.approx(1e8)
    assert bench.max_over_ranks(7.0, 1) == 7.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = SimpleNamespace(config=1, ranks=0, steps=1, warmup=0, gpus=2, ref_records=1e4)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
