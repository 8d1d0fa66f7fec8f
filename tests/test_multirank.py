"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1).

The sort does not shard (every rank sorts its own seeded inputs: replicas
only), so the multi-rank logic is the timing: each rank's time, the maximum
over ranks (the job ends with its slowest rank), and the whole-job throughput
from the keys of all ranks over that maximum.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import workloads  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 3.0 * (world - rank)]  # rank-dependent timings
        got = bench.max_over_ranks(torch, dist, times, "cpu")
        keys_per_rank = 5 * (1 << 20)
        value = bench.job_gkeys_per_s(world, keys_per_rank, got[0] / 1e3)
        # every rank draws its own inputs (seed = rank): nothing is exchanged
        own = workloads.generate("uniform", 4096, 16, seed=rank, stream=0)
        gathered = [torch.zeros(4096, dtype=torch.int32) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(own.astype("int32")))
        distinct = not torch.equal(gathered[0], gathered[1])
        out.put((rank, got, value, distinct))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    mp.start_processes(rank_main, args=(world, free_port(), out), nprocs=world, join=True, start_method="spawn")
    results = sorted(out.get(timeout=60) for _ in range(world))
    want_times = [10.0 + world - 1, 3.0 * world]  # element-wise maxima over the ranks
    for rank, got, value, distinct in results:
        assert got == want_times, (rank, got)
        # all ranks' keys over the slowest rank's time
        assert value == pytest.approx(world * 5 * (1 << 20) / (want_times[0] / 1e3) / 1e9)
        assert distinct  # the replicas sort different data


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(torch, None, [1.5, 2.0], "cpu") == [1.5, 2.0]
    assert bench.job_gkeys_per_s(1, 2_000_000_000, 2.0) == pytest.approx(1.0)
