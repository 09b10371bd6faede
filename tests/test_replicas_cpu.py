"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as
torchrun starts them) run replicas joined only by a barrier and a
max-over-ranks of their timings; the whole-job rate counts every rank's
units over the slowest rank's time.  The oracle reference arm runs on rank
0 alone; the other ranks exit at once."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _, pg = bench.dist_setup(backend="gloo")
    try:
        assert (w, r) == (world, rank)
        bench.barrier(pg)
        # rank r "took" 10 * (r + 1) ms for 1e6 units
        ms_max, rate = bench.replica_rate(pg, w, 1e6, 10.0 * (r + 1))
        out[rank] = (ms_max, rate)
        # the reference arm: rank 0 only (argument parsing is not needed
        # for the early exit of the other ranks)
        if r != 0:
            assert bench.run_reference(None, w, r, pg) == 0
    finally:
        pg.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world,
             join=True)
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        ms_max, rate = out[r]
        assert ms_max == 20.0
        assert rate == pytest.approx(world * 1e6 / 20e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")
           if k in os.environ}
    try:
        w, r, local, pg = bench.dist_setup()
        assert (w, r, local, pg) == (1, 0, 0, None)
        assert bench.replica_rate(None, 1, 5e5, 5.0) == (5.0, 1e8)
    finally:
        os.environ.update(env)
