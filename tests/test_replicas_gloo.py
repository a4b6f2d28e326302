"""Replica mode of the benchmark on two CPU ranks (gloo): every rank times its own copy of the
workload; the barrier pairs up the ranks and the reported time is the slowest rank's."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    bench.dist_init("gloo")
    assert bench.dist_env() == (rank, rank, world)
    bench.dist_barrier()
    got = bench.dist_max(0.5 + rank)             # rank r "measured" 0.5 + r
    bench.dist_barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_dist_max_over_two_ranks():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    assert res == {0: 1.5, 1: 1.5}, res


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE") if k in os.environ}
    try:
        assert bench.dist_env() == (0, 0, 1)
        assert bench.dist_max(3.25) == 3.25
        bench.dist_barrier()                     # no process group: nothing to wait for
    finally:
        os.environ.update(env)
