"""The multi-rank measurement logic of bench.py on CPU: two gloo ranks, each with its own step
time, gather every rank's time and report the whole-job throughput against the slowest rank
(the path shards by individuals with no data-path collective; the only collective is this
timing gather). Run as two spawned processes over 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per_rank = bench.gather_step_ms(times[rank], world, "cpu")
        value, slow = bench.aggregate(per_rank, 512)
        q.put((rank, per_rank, value, slow))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_times_and_aggregate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [2000.0, 2500.0]                 # ms per step on each rank
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, per_rank, value, slow in out:
        assert per_rank == times                               # every rank sees every time
        assert slow == 2500.0                                  # the job lasts as long as the slowest rank
        assert value == pytest.approx(2 * 512 / 2.5)           # both ranks' individuals / that time


def test_single_rank_needs_no_collective():
    import bench
    assert bench.gather_step_ms(1234.0, 1, "cpu") == [1234.0]
    assert bench.aggregate([1000.0], 512) == (512.0, 1000.0)
