"""Host logic of the N > 1 bench path on CPU: two gloo ranks, each timing an
independent replica; the job's time is the slowest rank's and its throughput
counts the units of every rank.  The reference arm runs on rank 0 only."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms_local = [12.0, 20.0][rank]      # rank 1 is the slower one
        ms_max, value = b.aggregate_ranks(ms_local, 1000, world, dist, torch.device("cpu"))
        out[rank] = (ms_max, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_units():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, value = res[r]
        assert ms_max == 20.0
        assert value == pytest.approx(1000 * world / 0.020)


def test_single_rank_needs_no_process_group():
    b = _bench()
    ms_max, value = b.aggregate_ranks(5.0, 300, 1, None, torch.device("cpu"))
    assert ms_max == 5.0 and value == pytest.approx(300 / 0.005)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    b = _bench()
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    args = b.parse()
    assert b.run_reference(args, rank=1, world=2) is None
