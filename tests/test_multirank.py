"""The N > 1 host path of bench.py (independent replicas, no data-path
collective) with two gloo ranks on the CPU: the timing is the slowest rank's
on every rank, throughput counts the solves of all ranks, and the reference
arm runs on rank 0 alone."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for its 10 solves
        sec = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        q.put((rank, sec, bench.weak_value(world, 10, sec)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [r for r, _, _ in got] == [0, 1]
    for _, sec, value in got:
        assert sec == 2.0                  # the slower rank's time on both
        assert value == pytest.approx(10.0)  # 2 ranks x 10 solves / 2 s
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.weak_value(1, 18, 0.5) == 36.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda rows: pytest.fail("rank 1 must not run the oracle"))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(bench.parse()) == 0
    assert capsys.readouterr().out == ""
