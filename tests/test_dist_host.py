"""Host logic of bench.py's N-rank runs on CPU: two gloo ranks on 127.0.0.1.
The query has no exchange step (independent replicas), so the only
cross-rank arithmetic is the timing and rate aggregation: the max over the
ranks' times, and the whole-job rate as world x the slowest rank's rate."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.dist_max(1.5 + rank, world)             # per-rank times 1.5, 2.5
        r = bench.dist_max_rate(10.0 * (rank + 1), world)  # per-rank rates 10, 20
        bench.barrier(world)
        one = bench.dist_max(7.0, 1)                       # world 1: no collective
        out.put((rank, t, r, one))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, r, one in got:
        assert t == 2.5   # the slowest rank's time on every rank
        assert r == 20.0  # world x the slowest rank's rate (2 x 10)
        assert one == 7.0
    assert [g[0] for g in got] == [0, 1]


def test_single_process_needs_no_process_group():
    import bench
    assert os.environ.get("WORLD_SIZE", "1") == "1" or pytest.skip("run under a launcher")
    world, rank, local = bench.dist_init(1)
    assert (world, rank, local) == (1, 0, 0)
    assert bench.dist_max(3.0, world) == 3.0 and bench.dist_max_rate(5.0, world) == 5.0
    bench.barrier(world)
