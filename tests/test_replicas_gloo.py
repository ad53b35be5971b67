"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would start
them, combine their timings into the whole-job rate.  Pairs are independent,
so the ranks are replicas: no data-path collective, only the max of the
timed-region times and the units of all ranks over it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.slowest_over_ranks(times[rank], "cpu")
        rate = bench.replica_rate(w, 4000 * 4, slowest * 1e-3)
        seeds = bench.replica_seeds(rank)
        dist.barrier()
        out.put((rank, slowest, rate, seeds))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_replicas_report_all_units_over_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [1180.0, 1234.5]   # ms of each rank's timed region
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    for rank, slowest, rate, seeds in res:
        assert slowest == max(times)
        assert rate == pytest.approx(world * 4000 * 4 / (max(times) * 1e-3))
    # every replica renders its own scenes
    assert res[0][3] != res[1][3] and set(res[0][3]).isdisjoint(res[1][3])


def test_single_rank_needs_no_process_group():
    assert not (dist.is_available() and dist.is_initialized())
    assert bench.slowest_over_ranks(12.5, "cpu") == 12.5
    assert bench.replica_rate(1, 100, 0.5) == 200.0
