"""The multi-rank (replica) path of bench.py on CPU with gloo, world size 2:
barrier, max over ranks of the timed region, and the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(dist, ms_local, device="cpu")
    value = bench.aggregate_mops(1000, 2, world, ms_max)
    out.put((rank, ms_max, value))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_replicas_take_max_over_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    # 2 ranks x 2 steps x 1000 ops in 15 ms
    assert res[0][2] == pytest.approx(2 * 2 * 1000 / 0.015 / 1e6)
