"""Host-side logic of the benchmark's multi-GPU path, as two gloo ranks on CPU:
the rank environment, the maximum of the per-rank times over the process group
(a job takes its slowest rank's time), and the whole-job throughput (weak
scaling: every rank adds its own scene). The GPU part of that path, one scene per
rank with no data-path collective, is what one rank runs alone."""
import os
import socket

import pytest

import bench


def free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        slowest = bench.max_over_ranks(1.5 + rank, w, "cpu")  # rank 1 is the slow one
        dist.barrier()
        q.put((rank, w, r, loc, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [x[:4] for x in res] == [(0, 2, 0, 0), (1, 2, 1, 1)]
    assert [x[4] for x in res] == [2.5, 2.5]


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25


def test_job_throughput_counts_every_rank():
    one = bench.job_throughput(1, 5, 256 ** 3, 8, 2.0)
    assert one == pytest.approx(5 * 256 ** 3 * 8 / 2.0)
    assert bench.job_throughput(4, 5, 256 ** 3, 8, 2.0) == pytest.approx(4 * one)
