"""The N>1 path of bench.py on CPU: two gloo ranks, each bounding its own pool
(weak scaling, no data-path collective); only the max-over-ranks timing is a
collective.  The pools are bounded by the oracle here (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.rank_pool(rank)
    m = bench.max_over_ranks(world, float(rank + 1) * 1.5)
    bench.barrier(world)
    q.put((rank, w.N, int((w.rows[:4].astype(np.int64) * np.arange(200)).sum()) + int(w.depths[:64].sum()), int(w.p.sum()), m))
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_gloo_ranks_get_distinct_pools_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, s0, p0, m0), (r1, n1, s1, p1, m1) = res
    assert n0 == n1 == 262144            # fixed work per rank: weak scaling
    assert p0 == p1                      # same instance on every rank
    assert s0 != s1                      # distinct pools
    assert m0 == m1 == 3.0               # max over ranks
