"""Batched persistent launch (many pools of many instances in one kernel) vs
the oracle and vs one plain launch per pool: bit-exact, alone and in the mix."""
import numpy as np
import pytest

import oracle
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def small_batch(seeds, max_nodes):
    """Instances of the batched workload's recipe (n from {20,50,100,200}, m
    from {5,10,20}), with pools cut to at most max_nodes nodes."""
    out = []
    for w in workloads.batched_instances(seeds):
        N = min(w.N, max_nodes)
        out.append(workloads.PoolWorkload(w.name, w.n, w.m, w.seed, w.p, w.rows[:N].copy(), w.depths[:N].copy()))
    return out


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batch_matches_oracle_and_plain_launches(gpu_lib):
    import torch
    fsp = gpu_lib
    ws = small_batch(range(100, 112), 700)
    insts = [fsp.Instance(w.p) for w in ws]
    bufs = [(dev(w.rows), dev(w.depths)) for w in ws]
    outs = [torch.full((w.N,), -7, dtype=torch.int32, device="cuda") for w in ws]
    pools = [(inst, r, d, o) for inst, (r, d), o in zip(insts, bufs, outs)]
    with fsp.Batch(pools) as b:
        q = b.query()
        assert q["nodes"] == sum(w.N for w in ws)
        b.launch()
        torch.cuda.synchronize()
        got = [o.cpu().numpy().copy() for o in outs]
        for o in outs:
            o.fill_(-7)
        b.launch_graph()
        b.launch_graph()
        torch.cuda.synchronize()
        got_graph = [o.cpu().numpy().copy() for o in outs]
    for w, inst, (r, d), g, gg in zip(ws, insts, bufs, got, got_graph):
        alone = fsp.fsp_bound_pool(inst, r, d)
        torch.cuda.synchronize()
        want = oracle.Tables(w.p).lb_pool(w.rows, w.depths, threads=16)
        assert np.array_equal(g, want), w.name
        assert np.array_equal(gg, want), w.name
        assert np.array_equal(alone.cpu().numpy(), want), w.name
    for inst in insts:
        inst.close()


def test_batch_with_empty_invalid_and_ragged_pools(gpu_lib):
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(9)
    specs = [(7, 5, 0), (33, 12, 45), (20, 20, 1), (64, 3, 97), (20, 20, 33)]
    insts, pools, ref = [], [], []
    for n, m, N in specs:
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
        if N > 3:
            depths[0] = -2          # invalid depth
            rows[1, :3] = [0, 0, 1]  # duplicate
            depths[1] = 3
        inst = fsp.Instance(p)
        insts.append(inst)
        out = torch.empty(N, dtype=torch.int32, device="cuda")
        pools.append((inst, dev(rows.reshape(N, n)), dev(depths), out))
        ref.append(oracle.Tables(p).lb_pool(rows.reshape(N, n), depths, threads=8))
    with fsp.Batch(pools, warps_per_block=3) as b:
        b.launch()
        torch.cuda.synchronize()
    for (inst, _, _, out), want in zip(pools, ref):
        assert np.array_equal(out.cpu().numpy(), want)
    for inst in insts:
        inst.close()


def test_batch_rejects_wide_instances(gpu_lib):
    import torch
    fsp = gpu_lib
    p = np.full((10, 4), 5000, np.int32)
    with fsp.Instance(p) as inst:
        r = torch.zeros((3, 10), dtype=torch.int16, device="cuda")
        d = torch.zeros(3, dtype=torch.int32, device="cuda")
        o = torch.empty(3, dtype=torch.int32, device="cuda")
        with pytest.raises(fsp.FspError):
            fsp.Batch([(inst, r, d, o)])


def test_full_batched_workload_sampled(gpu_lib):
    """The 64-instance batched workload (seeds 100-163, pools of 1,024 to
    65,536 nodes) in one graph launch; every pool is compared with its own
    plain launch, and a sample of nodes with the oracle."""
    import torch
    fsp = gpu_lib
    ws = workloads.batched_instances()
    insts = [fsp.Instance(w.p) for w in ws]
    bufs = [(dev(w.rows), dev(w.depths)) for w in ws]
    outs = [torch.empty(w.N, dtype=torch.int32, device="cuda") for w in ws]
    with fsp.Batch([(i, r, d, o) for i, (r, d), o in zip(insts, bufs, outs)]) as b:
        b.launch_graph()
        torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for w, inst, (r, d), o in zip(ws, insts, bufs, outs):
        got = o.cpu().numpy()
        alone = fsp.fsp_bound_pool(inst, r, d)
        torch.cuda.synchronize()
        assert np.array_equal(got, alone.cpu().numpy()), w.name
        idx = rng.choice(w.N, min(w.N, 64), replace=False)
        assert np.array_equal(got[idx], oracle.Tables(w.p).lb_pool(w.rows[idx], w.depths[idx], threads=16)), w.name
    for inst in insts:
        inst.close()


def test_batch_autotune_and_every_node_tile_agree(gpu_lib):
    """fsp_batch_autotune picks one of the timed node tiles; plans with 16, 8
    and 2 warps per block and the tuned one write the same bounds, equal to
    the oracle's."""
    import torch
    fsp = gpu_lib
    ws = small_batch(range(120, 128), 900)
    insts = [fsp.Instance(w.p) for w in ws]
    bufs = [(dev(w.rows), dev(w.depths)) for w in ws]
    outs = [torch.empty(w.N, dtype=torch.int32, device="cuda") for w in ws]
    pools = [(inst, r, d, o) for inst, (r, d), o in zip(insts, bufs, outs)]
    best_w, ms = fsp.fsp_batch_autotune(pools)
    assert best_w in (16, 12, 8, 6, 4, 2) and ms > 0
    wants = [oracle.Tables(w.p).lb_pool(w.rows, w.depths, threads=16) for w in ws]
    for W in (16, 8, 2, best_w):
        for o in outs:
            o.fill_(-7)
        with fsp.Batch(pools, warps_per_block=W) as b:
            assert b.query()["warps_per_block"] == W
            b.launch_graph()
            torch.cuda.synchronize()
        for o, want in zip(outs, wants):
            assert np.array_equal(o.cpu().numpy(), want), W
    for inst in insts:
        inst.close()


@pytest.mark.parametrize("cpi", [1, 32, 64, 96, 190])
def test_couple_sliced_batches_match_oracle(gpu_lib, cpi):
    """Plans split by couples (32 to 190 couples per work item, rounded up to
    whole groups of 32): pools of more groups are cut into slices that meet
    in an atomic max on zeroed bounds; pools of one group stay whole.  Mixed
    instances (m = 5, 12, 20, 27), invalid rows (every slice must agree on
    them), ragged and empty pools, per-job release times; plain and graph
    launches, the graph replayed twice; all equal to the oracle."""
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(700 + cpi)
    specs = [(40, 20, 700, 0), (33, 27, 333, 0), (23, 5, 90, 0), (70, 12, 257, 0), (20, 20, 0, 0),
             (50, 20, 401, fsp.FSP_INSTANCE_RELEASE_PER_JOB)]
    insts, pools, wants = [], [], []
    for n, m, N, flags in specs:
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
        if N > 60:
            depths[[3, 50]] = [-1, n + 1]
            rows[7, :2] = [5, 5]
            depths[7] = max(int(depths[7]), 2)
        inst = fsp.Instance(p, flags=flags)
        insts.append(inst)
        pools.append((inst, dev(rows.reshape(N, n)), dev(depths), torch.full((N,), -7, dtype=torch.int32,
                                                                               device="cuda")))
        rel = oracle.RELEASE_EST if flags else oracle.RELEASE_HEADS
        wants.append(oracle.Tables(p).lb_pool(rows.reshape(N, n), depths, threads=16, release=rel))
    with fsp.Batch(pools, warps_per_block=4, couples_per_item=cpi) as b:
        assert b.query()["couples_per_item"] == cpi
        b.launch()
        torch.cuda.synchronize()
        for (_, _, _, o), want in zip(pools, wants):
            assert np.array_equal(o.cpu().numpy(), want), cpi
            o.fill_(-7)
        b.launch_graph()
        b.launch_graph()
        torch.cuda.synchronize()
        for (_, _, _, o), want in zip(pools, wants):
            assert np.array_equal(o.cpu().numpy(), want), cpi
    for inst in insts:
        inst.close()


def test_batch_autotune_ex_picks_tile_and_couple_split(gpu_lib):
    """fsp_batch_autotune_ex returns one of the timed (warps, couples per
    item) pairs, and the plan it picks writes the oracle's bounds."""
    import torch
    fsp = gpu_lib
    ws = small_batch(range(130, 136), 600)
    insts = [fsp.Instance(w.p) for w in ws]
    outs = [torch.empty(w.N, dtype=torch.int32, device="cuda") for w in ws]
    pools = [(inst, dev(w.rows), dev(w.depths), o) for inst, w, o in zip(insts, ws, outs)]
    W, cpi, ms = fsp.fsp_batch_autotune_ex(pools)
    assert W in (16, 12, 8, 6, 4, 2) and cpi in (0, 32, 64, 96, 128) and ms > 0
    for o in outs:
        o.fill_(-7)
    with fsp.Batch(pools, warps_per_block=W, couples_per_item=cpi) as b:
        b.launch_graph()
        torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        assert np.array_equal(o.cpu().numpy(), oracle.Tables(w.p).lb_pool(w.rows, w.depths, threads=16))
    for inst in insts:
        inst.close()


@pytest.mark.parametrize("W", [0, 3, 16])
def test_few_couple_instances_in_one_plan_match_oracle(gpu_lib, W):
    """Instances with few couples (m = 2 .. 12, one group of 32 couple lanes
    or two) beside one with six groups (m = 20) in one plan: pools of ragged
    sizes, an empty one, invalid rows at every 32-node boundary of the first
    128 nodes, per-job release times; automatic and fixed node tiles, and the
    same pools in a couple-sliced plan, must all match the oracle bit for
    bit."""
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(77)
    specs = [(9, 2, 300), (12, 3, 257), (15, 4, 33), (20, 5, 1000), (25, 6, 129), (18, 8, 200), (30, 10, 999),
             (22, 12, 513), (40, 20, 300), (16, 5, 0), (20, 5, 97)]
    ws, insts = [], []
    for i, (n, m, N) in enumerate(specs):
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
        if N > 130:
            for x in (0, 31, 32, 63, 64, 95, 96, 127, 128):  # both ends of the first 32-node batches
                depths[x] = -1 if x % 2 else n + 1
        release = i == len(specs) - 1
        ws.append((p, rows, depths, release))
        insts.append(fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB if release else 0))
    bufs = [(dev(r), dev(d)) for _, r, d, _ in ws]
    outs = [torch.full((r.shape[0],), -7, dtype=torch.int32, device="cuda") for _, r, _, _ in ws]
    pools = [(inst, r, d, o) for inst, (r, d), o in zip(insts, bufs, outs)]
    with fsp.Batch(pools, warps_per_block=W) as b:
        b.launch()
        torch.cuda.synchronize()
    for (p, rows, depths, release), o in zip(ws, outs):
        want = oracle.Tables(p).lb_pool(rows, depths, threads=8,
                                        release=oracle.RELEASE_EST if release else oracle.RELEASE_HEADS)
        assert np.array_equal(o.cpu().numpy(), want), (p.shape, rows.shape)
    # a couple-sliced plan agrees
    outs2 = [torch.full_like(o, -7) for o in outs]
    with fsp.Batch([(inst, r, d, o) for inst, (r, d), o in zip(insts, bufs, outs2)], warps_per_block=4,
                   couples_per_item=32) as b:
        b.launch()
        torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    for inst in insts:
        inst.close()
