"""Host logic of bench.py's multi-rank path, on CPU with gloo and two ranks.

A single chain does not shard (sweeps visit sites one after another), so
N GPUs run N independent windows: the whole-job value is N times one
window's flops over the slowest rank's time, and only rank 0 reports.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                # rank 1 is the slow replica
        slowest = bench.max_over_ranks(local_ms, world, "cpu")
        value = bench.replica_value(2.0e9, world, slowest)
        # the reference arm runs on rank 0 only; other ranks return nothing
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "cpu_sample_s": 0.0})()) \
            if rank != 0 else "skipped"
        out[rank] = (slowest, value, ref)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        slowest, value, ref = out[r]
        assert slowest == 15.0
        assert value == pytest.approx(2.0e9 * 2 / 15e-3 / 1e12)
    assert out[1][2] is None


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_value(1e12, 1, 1000.0) == pytest.approx(1.0)
