"""bench.py's multi-rank plumbing on CPU: world-size-2 gloo ranks, barrier,
max-over-ranks timing and whole-job aggregation (replicas only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank), RECOGS_DIST_BACKEND="gloo")
    import bench
    r, w, l = bench.dist_init()
    assert (r, w, l) == (rank, world, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    out[rank] = (mx, bench.aggregate_value(100, w, mx))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    mx, val = out[0]
    assert mx == 15.0
    assert val == pytest.approx(100 * 2 / 0.015)


def test_aggregate_single():
    import bench
    assert bench.aggregate_value(10, 1, 1000.0) == pytest.approx(10.0)
