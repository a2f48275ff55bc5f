"""The multi-rank (N > 1) host logic of bench.py on CPU, with two gloo ranks:
the whole-job figures take the slowest rank's time and the sum of all
ranks' points, each rank tracks its own streams (replicas, no exchange on
the data path), and the reference arm runs on rank 0 only."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        times, counts = bench.combine_ranks([10.0 + rank, 1.0 - rank * 0.5], [100.0 * (rank + 1), 7.0],
                                            "cpu")
        q.put((rank, times, counts))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_ranks_combine_max_time_and_total_points():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, times, counts in res:
        assert times == [11.0, 1.0]          # max over ranks
        assert counts == [300.0, 14.0]       # sum over ranks


def test_ranks_track_disjoint_streams():
    sys.path.insert(0, ROOT)
    import bench
    # rank r of a run with S streams per rank tracks streams r*S .. r*S+S-1
    (a,), (b,) = bench.make_streams(1, 0), bench.make_streams(1, 1)
    assert a.size != b.size or not (a.frame0 == b.frame0).all()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda *a: called.append(a) or {})
    bench.main()
    assert not called and capsys.readouterr().out == ""
