"""The multi-rank path on CPU: two gloo ranks, each with its own seeded points,
a max-reduction of the timings and the whole-job throughput (no GPU)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from inputs import workloads as wl
    from paper_1712_08226_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = wl.workload_random10(64, seed_pts=shard.rank_point_seed(rank))["x"]
    local_t = np.array([1.0 + rank, 5.0 - rank])
    red = shard.reduce_max(local_t, dist)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, x.sum(), red.tolist(), x[:2].tolist()))


def test_two_gloo_ranks_shard_points_and_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(2):
        r, s, red, head = q.get(timeout=120)
        res[r] = (s, red, head)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from inputs import workloads as wl
    from paper_1712_08226_gb300 import shard
    # rank 0 solves the standard point set, rank 1 a different one
    std = wl.workload_random10(64)["x"]
    assert np.allclose(res[0][2], std[:2])
    assert not np.allclose(res[0][2], res[1][2])
    # both ranks see the element-wise maximum of the timings
    assert res[0][1] == res[1][1] == [2.0, 5.0]
    assert shard.job_throughput(100, 2, 0.5) == 400.0
