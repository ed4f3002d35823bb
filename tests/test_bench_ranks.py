"""Host-side multi-rank logic of bench.py on CPU with the gloo backend (world size 2): the
timed value is the maximum over ranks on every rank, and the reference arm does its work on
rank 0 only (the other ranks return at once)."""
import os
import socket
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    values = [3.25, 7.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), values, out), nprocs=world, join=True,
                           start_method="spawn")
        assert dict(out) == {0: 7.5, 1: 7.5}


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_samples", lambda *a, **k: called.append(1))
    args = types.SimpleNamespace(n=128, warmup=3, steps=5, gpus=2)
    assert bench.run_reference(args) == 0
    assert not called and capsys.readouterr().out == ""
