"""The N > 1 path of bench.py (replicas only: one independent mapping step per
GPU, no collective on the data path) on CPU with the gloo backend and two
ranks: the per-rank times reduce to the slowest rank's, the whole-job rate
counts every replica's iterations, and the reference arm runs on rank 0
alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_ms = [2.0, 3.5][rank]
    slowest = bench.max_over_ranks(per_rank_ms, "cpu")
    out.put((rank, slowest, bench.job_rate(slowest, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_both_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 3.5
        assert rate == pytest.approx(2 * 1000.0 / 3.5)


def test_without_a_process_group_the_value_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.job_rate(2.0, 1) == 500.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        gpus, steps, warmup, ref_rows = 2, 1, 3, 64
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(Args())  # returns before any oracle work
    assert capsys.readouterr().out == ""
