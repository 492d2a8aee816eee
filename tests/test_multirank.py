"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs its own stream (distinct seeds, no data-path collective), the timed
region's duration is the slowest rank's, and the whole-job rate counts the
units of all ranks."""
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


def _worker(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]
        ms = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        rate = bench.whole_job_rate(16 * 10, ms / 1e3, world)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(0, rank))
        q.put((rank, ms, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, seeds in out:
        assert ms == 150.0                        # the slowest rank
        assert rate == pytest.approx(2 * 160 / 0.150)
        assert len(set(seeds)) == 2               # independent streams
