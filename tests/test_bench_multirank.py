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


def _run_bench(args, env_extra):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "bench.py"] + args, cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    return lines


def test_reference_arm_prints_one_contract_line_on_rank_zero_only():
    """The reference arm (the CPU oracle on one individual of the benchmark batch) prints one
    JSON line with the contract's keys on rank 0 and nothing on the other ranks."""
    lines = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-threads", "2"],
                       {"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "predictions/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    for key in ("metric", "ms_per_step", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "predictions/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"}) == []
