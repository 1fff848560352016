"""The bench's multi-rank host path on two CPU ranks (gloo): barrier, the
max-over-ranks job time and the whole-job weak-scaling aggregate."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist

    class A:
        pass
    w, r, _ = bench.dist_setup(A())
    bench.barrier(w)
    # rank r took (r + 1) * 100 ms for 2 steps of 160 units
    value, ms = bench.aggregate(160, 2, (r + 1) * 100.0, w)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, value, ms))


def test_two_gloo_ranks_aggregate_with_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, ms in res:
        assert w == world
        assert ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 160 * 2 / 0.2)
