"""Multi-process host logic of bench.py on CPU ranks (gloo, world size 2):
replicas share nothing but the final max-over-ranks of their step times, and
independent problems are dealt to ranks without a collective."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        out[rank] = (bench.max_over_ranks(10.0 + 5.0 * rank), bench.shard(7, rank, world))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_sharding_world2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                    # slowest rank's time
    assert sorted(res[0][1] + res[1][1]) == list(range(7))    # every problem once
    assert set(res[0][1]).isdisjoint(res[1][1])


def test_single_process_falls_back_to_local_value():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert [len(bench.shard(10, r, 4)) for r in range(4)] == [3, 3, 2, 2]
