"""bench.py's multi-rank path on CPU: two gloo ranks (one per process, as
torchrun launches them) meet at the barrier and report the whole-job
throughput over the slowest rank's time (replicas, weak scaling)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    local_ms = [120.0, 150.0][rank]          # rank 1 is the slow one
    value, ms_per_step, t_ms = bench.aggregate(local_ms, 30, world)
    bench.barrier(world)
    q.put((rank, value, ms_per_step, t_ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_over_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_per_step, t_ms in out:
        assert t_ms == 150.0                      # max over ranks
        assert ms_per_step == pytest.approx(5.0)
        assert value == pytest.approx(2 * 30 / 0.150)   # all steps of all ranks / slowest time


def test_single_rank_aggregate_is_local():
    import bench
    value, ms_per_step, t_ms = bench.aggregate(200.0, 50, 1)
    assert (value, ms_per_step, t_ms) == (pytest.approx(250.0), pytest.approx(4.0), 200.0)
