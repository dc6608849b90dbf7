"""Multi-rank logic of bench.py on CPU: two gloo processes check the
max-over-ranks time, the summed eigenpair count and the whole-job
throughput formula used when every rank solves its own replica."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    bench.barrier(ws)
    ms = [1000.0, 1500.0][rank]  # rank 1 is the slowest
    conv = [109, 107][rank]
    q.put((rank, bench.max_over_ranks(ms, ws), bench.sum_over_ranks(conv, ws), bench.throughput(conv, ms, ws)))
    dist.destroy_process_group()


def test_bench_rank_reductions_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, thr in out:
        assert mx == 1500.0 and sm == 216.0
        assert abs(thr - 216.0 / 1.5) < 1e-12


def test_reference_arm_only_rank0_reports(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        side, steps, warmup, cpu_sample_seconds = 64, 1, 3, 1.0

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
