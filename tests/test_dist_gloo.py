"""Host logic of the N > 1 benchmark path on two gloo ranks (CPU, no GPU).

bench.py runs one replica of the workload per rank ("replicas only": a
single factorization is not split across GPUs); the job time is the
slowest rank's time and the value is the work of all ranks over it.  The
reference arm runs on rank 0 alone and the other ranks exit 0 without work.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], dist)
        out[rank] = (ms, bench.aggregate_value(2.0e12, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    times = [1.5, 4.0]
    mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 4.0                                  # slowest replica
        assert value == pytest.approx(2.0e12 * 2 / 4.0e-3 / 1e12)   # both replicas' work


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.aggregate_value(1e12, 1, 1.0) == pytest.approx(1000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda *a, **k: called.append(1) or 0)
    assert bench.main() == 0
    assert called == []
