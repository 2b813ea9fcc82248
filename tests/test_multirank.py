"""The replica (N > 1) path of bench.py on CPU: two gloo ranks.

Under torchrun every rank runs an independent replica (its own seeded
system) and rank 0 reports the whole-job value from the slowest rank's time
and the summed counters.  These tests run the rank-combination helpers of
bench.py in two processes over gloo on 127.0.0.1 (no GPU), and check that the
reference arm does no work on ranks other than 0.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    import bench
    cpu = torch.device("cpu")
    w, r, local = bench._dist()
    t_rank = 1.0 + rank             # rank 1 is the slow one
    t_max = bench._reduce(t_rank, w, cpu, "max")
    total = bench._reduce(10.0 * (rank + 1), w, cpu, "sum")
    bench._barrier(w)
    value = w * bench.ns_per_day(100, t_max)
    out[rank] = (w, r, t_max, total, value)
    dist.destroy_process_group()


def test_two_ranks_combine_like_the_bench():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        w, r, t_max, total, value = res[rank]
        assert (w, r) == (ws, rank)
        assert t_max == 2.0                       # the slowest rank's time
        assert total == 30.0                      # counters summed over ranks
        # whole-job throughput: N replicas' steps over the slowest rank's time
        assert abs(value - 2 * (100 * 1e-6 * 86400 / 2.0)) < 1e-12


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup = 1, 3
    bench.reference_arm(A())                      # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
