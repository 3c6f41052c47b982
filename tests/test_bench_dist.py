"""The benchmark's multi-process path (barrier, max / sum over ranks) on CPU
with the gloo backend, world size 2."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 1.5 + r)
    sm = bench.sum_over_ranks(dist, 10.0 * (r + 1))
    out.put((r, mx, sm))
    dist.destroy_process_group()


def test_replica_aggregation_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.5, 30.0), (1, 2.5, 30.0)]


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(None, 3.0) == 3.0
    assert bench.sum_over_ranks(None, 4.0) == 4.0
