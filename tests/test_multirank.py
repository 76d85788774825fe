"""The benchmark's multi-process host logic on CPU with the gloo backend (world size 2):
each rank reports its own timed interval, the job rate uses the slowest rank, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seconds = 1.0 + rank          # rank 1 is the slow one
        out[rank] = (bench.max_over_ranks(seconds), bench.whole_job_rate(5, seconds, world), bench.dist_env())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_rate_uses_slowest_rank_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        mx, rate, env = out[rank]
        assert mx == 2.0
        assert rate == pytest.approx(5 * world / 2.0)
        assert env == (world, rank, rank)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(4, 2.0, 1) == 2.0


def test_reference_arm_only_on_rank0(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.main()   # rank 1 returns without work and prints nothing
    assert capsys.readouterr().out == ""
