"""The multi-rank path of bench.py on CPU: two gloo ranks, each one replica
of the workload; the job's time is the slowest rank's and its throughput
counts both ranks' work."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    m = bench.reduce_max(ms, world)
    v = bench.aggregate(8e9, m, world)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    m, v = res[0]
    assert m == 150.0
    assert v == pytest.approx(2 * 8e9 / 0.150 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(1e9, 1000.0, 1) == pytest.approx(1.0)
