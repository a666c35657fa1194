"""The bench's N > 1 path on the CPU: world_size 2 over gloo.

Each rank runs the whole workload (replicas); the job's time is the slowest
rank's, the value counts the units of every rank.  The reference arm runs on
rank 0 only."""
import argparse
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, q):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tdist.barrier()
        mx = bench.reduce_max_ms(local_ms[rank], tdist, "cpu")
        q.put((rank, mx, bench.job_value(world, 3, 2.0e9, mx)))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [10.0, 25.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, mx, val in got:
        assert mx == 25.0
        # 2 ranks x 3 steps x 2e9 units in 25 ms
        assert val == pytest.approx(2 * 3 * 2.0e9 / 0.025 / 1e9)


def test_single_rank_needs_no_group():
    import bench
    assert bench.reduce_max_ms(7.5, None, "cpu") == 7.5
    assert bench.job_value(1, 4, 1e9, 100.0) == pytest.approx(40.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(rows=1000, steps=1, warmup=1, gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
