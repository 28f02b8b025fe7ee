"""Host-side logic of the multi-GPU (replica) bench path on CPU: two gloo
ranks on 127.0.0.1 agree on the largest per-rank time, the whole-job value
counts every rank's work, and only rank 0 of the reference arm prints."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist           # noqa: E402
import torch.multiprocessing as mp         # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench                                # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        dist.barrier()
        out[rank] = bench.max_over_ranks(ms, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 15.0
    # weak scaling: every rank's units count
    assert bench.whole_job_value(1000, 4, world, out[0]) == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(100, 2, 1, 10.0) == pytest.approx(20000.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.reference_arm(bench.parse())
    assert capsys.readouterr().out == ""
