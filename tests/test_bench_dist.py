"""The multi-rank path of bench.py on CPU: two gloo ranks, barrier and the
max-over-ranks timing that turns per-rank work into a whole-job rate (weak
scaling: every rank runs its own replica of the workload)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    local = 2.0 + rank  # rank 1 is the slow one
    total_s, value = bench.aggregate(w, 1e9, 3, local)
    out.put((rank, total_s, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_by_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_s, value in res:
        assert total_s == pytest.approx(3.0)
        assert value == pytest.approx(2 * 1e9 * 3 / 3.0)


def test_reference_arm_ranks_other_than_zero_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 1, "config": "c2"})()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
