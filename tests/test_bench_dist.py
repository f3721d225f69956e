"""Host-side logic of the multi-process bench path on CPU (gloo, 2 ranks):
timing reduction over ranks and the whole-group sharding helper."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r = bench.init_dist("gloo")
    out = {
        "ws": ws,
        "max": bench.reduce_scalar(10.0 * (rank + 1), "max"),
        "sum": bench.reduce_scalar(rank + 1.0, "sum"),
        "shard": bench.shard_signals(1000, world, rank, 16),
    }
    bench.barrier()
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_rank_reduction_and_sharding():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["ws"] == world
        assert res[r]["max"] == 20.0
        assert res[r]["sum"] == 3.0
    (a0, a1), (b0, b1) = res[0]["shard"], res[1]["shard"]
    assert a0 == 0 and a1 == b0 and b1 == 1000
    assert a1 % 16 == 0            # shards hold whole checksum groups


def test_single_process_helpers_are_identity():
    import bench
    assert bench.reduce_scalar(3.5, "max") == 3.5
    assert bench.shard_signals(100, 1, 0, 16) == (0, 100)
    assert bench.flops(1024, 2) == pytest.approx(5 * 1024 * 10 * 2)
