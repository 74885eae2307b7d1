"""Multi-rank logic of bench.py on CPU: two gloo ranks, each timing its own
independent replica; the whole-job value is all ranks' cell-updates over
the slowest rank's time, and the reference arm prints on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_max, value = bench.aggregate_ranks(ms[rank], 1000.0, torch.device("cpu"))
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_takes_slowest_rank():
    world, ms = 2, [40.0, 50.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms_max, value in out:
        assert ms_max == 50.0
        assert value == pytest.approx(world * 1000.0 / 0.050)


def test_single_process_aggregation():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.aggregate_ranks(20.0, 1000.0, torch.device("cpu"))
    assert ms_max == 20.0 and value == pytest.approx(1000.0 / 0.020)


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1"])
    a = bench.parse()
    bench.main_reference(a)
    assert capsys.readouterr().out == ""
