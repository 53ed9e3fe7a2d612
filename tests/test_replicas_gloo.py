"""N > 1 replicas of the benchmark, host side: two gloo ranks on the CPU.

Each rank runs its own copy of the workload (no data-path collective); the job
time is the slowest rank's, the job rate sums the ranks' units, and only rank 0
of the reference arm runs and prints."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank)          # rank 1 is the slower replica
        rate = bench.job_rate(512 ** 3, ms, world)
        # the reference arm: ranks other than 0 leave at once, without output
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": world})())
        dist.barrier()
        q.put((rank, ms, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank_and_sum_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, rate, out in got:
        assert ms == 15.0                                       # max over ranks on every rank
        assert abs(rate - 2 * 512 ** 3 / 15e-3) < 1e-6 * rate   # both replicas' voxels
        if rank != 0:
            assert out == ""


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(100, 1000.0, 1) == 100.0
