"""GPU bounding vs the CPU oracle, element by element (bit-exact: integer).

All inputs are seeded synthetic pools from paper_1208_3933_gb300.workloads;
every call goes through the C ABI (fsp_bound_pool / _ex / _host).
"""
import numpy as np
import pytest

import oracle
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu

THREADS = 16


def to_dev(rows, depths):
    import torch
    return torch.from_numpy(np.ascontiguousarray(rows)).cuda(), torch.from_numpy(np.ascontiguousarray(depths)).cuda()


def gpu_bounds(fsp, inst, rows, depths, config=None, stream=None):
    import torch
    r, d = to_dev(rows, depths)
    out = fsp.fsp_bound_pool(inst, r, d, config=config, stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_bounds(p, rows, depths):
    return oracle.Tables(p).lb_pool(rows, depths, threads=THREADS)


def pool(seed, n, m, N, hi=99):
    rng = np.random.default_rng(seed)
    p = rng.integers(1, hi + 1, size=(n, m), dtype=np.int32)
    rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
    return p, rows, depths


@pytest.mark.parametrize("n,m,N", [(20, 20, 5000), (50, 10, 3001), (200, 20, 1500), (7, 5, 999),
                                   (1, 2, 3), (2, 2, 50), (13, 32, 700), (100, 3, 1111)])
def test_pool_matches_oracle(gpu_lib, n, m, N):
    fsp = gpu_lib
    p, rows, depths = pool(n * 1000 + m, n, m, N)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths)
    want = oracle_bounds(p, rows, depths)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("bps", [1, 2])
@pytest.mark.parametrize("ppt", [0, 1, 7])
def test_every_lockstep_shape_matches_oracle(gpu_lib, K, bps, ppt):
    """Node-lockstep kernel, explicit shapes, including couple tiles of 1 and
    7 couples (190 couples at m=20), which force re-staging of the tables for
    every node tile and a ragged last tile."""
    fsp = gpu_lib
    p, rows, depths = pool(77, 40, 20, 3 * 128 * K + 17)
    cfg = dict(kernel=fsp.FSP_KERNEL_LOCKSTEP, nodes_per_thread=K, blocks_per_sm=bps, pairs_per_tile=ppt)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    assert np.array_equal(got, oracle_bounds(p, rows, depths))


@pytest.mark.parametrize("W", [1, 3, 16])
@pytest.mark.parametrize("staging,positions", [(1, 0), (2, 0), (2, 4), (2, 12), (2, 64), (3, 0), (3, 4), (3, 64),
                                               (4, 0), (4, 4), (4, 12)])
@pytest.mark.parametrize("nm", [(40, 20), (23, 9), (17, 5), (70, 12), (33, 27)])
def test_every_lanes_shape_matches_oracle(gpu_lib, W, staging, positions, nm):
    """Couple-lanes kernel, explicit shapes: 1 to 16 warps per block; records
    resident (warps claim batches independently), streamed with Johnson
    positions staged 4, 12 or 64 at a time (re-staging, ragged last chunk),
    split into prep and scan kernels, or streamed per warp; couple counts
    below, at and above one warp of 32 (m = 5, 9, 12, 20, 27)."""
    fsp = gpu_lib
    n, m = nm
    p, rows, depths = pool(78 + n, n, m, 2 * 32 * W * 3 + 19)
    if staging == 4 and W == 16 and positions > 4:
        positions = 4  # sixteen rings of larger tiles exceed a block's shared memory
    cfg = dict(kernel=fsp.FSP_KERNEL_LANES, warps_per_block=W, positions_per_tile=positions, staging=staging)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    assert np.array_equal(got, oracle_bounds(p, rows, depths))


@pytest.mark.parametrize("staging", [2, 3])
@pytest.mark.parametrize("ppt", [32, 64, 96, 160])
@pytest.mark.parametrize("W,positions", [(1, 12), (4, 12), (3, 0)])
@pytest.mark.parametrize("nm", [(40, 20), (70, 12), (33, 27), (23, 9)])
def test_couple_sliced_work_items_match_oracle(gpu_lib, ppt, W, positions, nm, staging):
    """Streamed staging with every block batch split by couples over several
    work items (pairs_per_tile 32 to 160: one to five groups of 32 couples per
    item, the last slice ragged or a single group), the slices combined by
    atomic max into zeroed bounds; positions staged 12 at a time (tiles
    re-staged within and across items) or in whole groups.  Invalid rows in
    the pool: every slice must agree on them."""
    fsp = gpu_lib
    n, m = nm
    p, rows, depths = pool(500 + n + m, n, m, 3 * 32 * W * 4 + 21)
    depths[[3, 50]] = [-1, n + 1]
    rows[7, :2] = [5, 5]
    depths[7] = max(int(depths[7]), 2)
    if staging == 3 and positions == 0:
        positions = 64  # split staging tiles positions
    cfg = dict(kernel=2, warps_per_block=W, positions_per_tile=positions, staging=staging, pairs_per_tile=ppt)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    want = oracle_bounds(p, rows, depths)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert got[3] == got[50] == got[7] == fsp.FSP_LB_INVALID


@pytest.mark.parametrize("ppt", [0, 32, 64, 160, 1000])
@pytest.mark.parametrize("W,bps", [(1, 0), (4, 0), (3, 5), (16, 1)])
@pytest.mark.parametrize("nm", [(40, 20), (70, 12), (33, 27), (23, 9), (200, 20)])
def test_global_staging_matches_oracle(gpu_lib, ppt, W, bps, nm):
    """Global staging: no shared-memory record tiles, every warp reads its
    couples' records through the register ring and takes its own work items
    (a 32-node batch and a couple slice: one to five groups of 32 couples,
    the last slice ragged, or all couples; 0 = slices chosen from the pool
    size); pools of a few warps' worth up to several per warp of the grid,
    with a ragged last batch and invalid rows that every slice must agree
    on."""
    fsp = gpu_lib
    n, m = nm
    p, rows, depths = pool(700 + n + m, n, m, 32 * W * 7 + 19)
    depths[[3, 50]] = [-1, n + 1]
    rows[7, :2] = [5, 5]
    depths[7] = max(int(depths[7]), 2)
    cfg = dict(kernel=2, staging=5, warps_per_block=W, blocks_per_sm=bps, pairs_per_tile=ppt)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    want = oracle_bounds(p, rows, depths)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert got[3] == got[50] == got[7] == fsp.FSP_LB_INVALID


@pytest.mark.parametrize("npw", [28, 56])
@pytest.mark.parametrize("ppt", [0, 32, 96, 1000])
@pytest.mark.parametrize("W,bps,positions", [(1, 0, 12), (4, 2, 0), (3, 1, 64), (6, 1, 96)])
@pytest.mark.parametrize("nm", [(40, 20), (70, 12), (33, 27), (23, 9), (200, 20)])
def test_28_node_sets_per_warp_match_oracle(gpu_lib, npw, ppt, W, bps, positions, nm):
    """Streamed staging with one or two sets of 28 nodes per warp (flag bits
    7, 15, 23 and 31 unused): block batches of npw W nodes with a ragged last
    batch, couple slices (0 = chosen from the pool size) combined by atomic
    max, record tiles of 12, 64 or 96 positions or whole groups, and invalid
    rows in either set."""
    fsp = gpu_lib
    n, m = nm
    p, rows, depths = pool(900 + n + m, n, m, npw * W * 5 + 23)
    depths[[3, 50, 40]] = [-1, n + 1, n + 2]
    rows[7, :2] = [5, 5]
    depths[7] = max(int(depths[7]), 2)
    cfg = dict(kernel=2, staging=2, nodes_per_thread=npw, warps_per_block=W, blocks_per_sm=bps,
               positions_per_tile=positions, pairs_per_tile=ppt)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    want = oracle_bounds(p, rows, depths)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert got[3] == got[50] == got[40] == got[7] == fsp.FSP_LB_INVALID


def test_two_node_sets_depth_order_release_and_refusals(gpu_lib):
    """56 nodes per warp on a depth-ordered pool (n >= 64, N >= 8,192) and with
    per-job release times; refused with 128-bit records and outside streamed
    staging."""
    fsp = gpu_lib
    w = workloads.named_pool("pool_200x20", N=9000)
    idx = np.random.default_rng(6).choice(w.N, 300, replace=False)
    two = dict(kernel=2, staging=2, nodes_per_thread=56, warps_per_block=4, blocks_per_sm=2, positions_per_tile=96)
    with fsp.Instance(w.p) as inst:
        a = gpu_bounds(fsp, inst, w.rows, w.depths, config=two)
        b = gpu_bounds(fsp, inst, w.rows, w.depths, config=dict(kernel=2, staging=2, warps_per_block=8))
        c = gpu_bounds(fsp, inst, w.rows, w.depths, config=dict(two, nodes_per_thread=28))
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.array_equal(a[idx], oracle_bounds(w.p, w.rows[idx], w.depths[idx]))
        r, d = to_dev(w.rows[:100], w.depths[:100])
        for bad in (dict(two, staging=1), dict(two, staging=3), dict(two, staging=5), dict(two, nodes_per_thread=40),
                    dict(two, tail_slices=2), dict(two, nodes_per_thread=28, staging=3)):
            with pytest.raises(fsp.FspError):
                fsp.fsp_bound_pool(inst, r, d, config=bad)
    with fsp.Instance(w.p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        got = gpu_bounds(fsp, inst, w.rows[:3000], w.depths[:3000], config=two)
    want = oracle.Tables(w.p).lb_pool(w.rows[:3000], w.depths[:3000], threads=THREADS, release=oracle.RELEASE_EST)
    assert np.array_equal(got, want)
    p, rows, depths = pool(9, 45, 11, 170, hi=20000)
    with fsp.Instance(p) as inst:
        r, d = to_dev(rows, depths)
        with pytest.raises(fsp.FspError):
            fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=2, nodes_per_thread=56, warps_per_block=2,
                                                       positions_per_tile=8))


def test_global_staging_depth_order_release_and_refusals(gpu_lib):
    """Global staging on a depth-ordered pool (n >= 64, N >= 8,192), sliced
    and whole, with per-job release times; refused for 128-bit records and
    for shapes outside its limits."""
    fsp = gpu_lib
    w = workloads.named_pool("pool_200x20", N=9000)
    idx = np.random.default_rng(5).choice(w.N, 300, replace=False)
    with fsp.Instance(w.p) as inst:
        a = gpu_bounds(fsp, inst, w.rows, w.depths, config=dict(kernel=2, staging=5, pairs_per_tile=64))
        b = gpu_bounds(fsp, inst, w.rows, w.depths, config=dict(kernel=2, staging=5, warps_per_block=8,
                                                                pairs_per_tile=190))
        c = gpu_bounds(fsp, inst, w.rows, w.depths, config=dict(kernel=2, staging=2, warps_per_block=8))
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.array_equal(a[idx], oracle_bounds(w.p, w.rows[idx], w.depths[idx]))
        r, d = to_dev(w.rows[:100], w.depths[:100])
        for bad in (dict(kernel=2, staging=5, warps_per_block=8, blocks_per_sm=3),
                    dict(kernel=2, staging=5, positions_per_tile=8), dict(kernel=2, staging=5, tail_slices=2)):
            with pytest.raises(fsp.FspError):
                fsp.fsp_bound_pool(inst, r, d, config=bad)
    with fsp.Instance(w.p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        got = gpu_bounds(fsp, inst, w.rows[:3000], w.depths[:3000], config=dict(kernel=2, staging=5,
                                                                                  warps_per_block=2))
    want = oracle.Tables(w.p).lb_pool(w.rows[:3000], w.depths[:3000], threads=THREADS, release=oracle.RELEASE_EST)
    assert np.array_equal(got, want)
    p, rows, depths = pool(9, 45, 11, 170, hi=20000)
    with fsp.Instance(p) as inst:
        assert inst.info().compact == 0
        r, d = to_dev(rows, depths)
        with pytest.raises(fsp.FspError):
            fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=5))


def test_couple_slices_with_depth_order_release_and_wide_records(gpu_lib):
    """Couple slices on a depth-ordered pool (n >= 64, N >= 8,192), with
    per-job release times, and with 128-bit records; the default shape of a
    small pool splits batches by couples and matches the unsplit shape."""
    import torch
    fsp = gpu_lib
    w = workloads.named_pool("pool_200x20", N=9000)
    sliced = dict(kernel=2, warps_per_block=8, positions_per_tile=96, staging=2, pairs_per_tile=64)
    whole = dict(sliced, pairs_per_tile=190, blocks_per_sm=2)
    idx = np.random.default_rng(4).choice(w.N, 300, replace=False)
    with fsp.Instance(w.p) as inst:
        a = gpu_bounds(fsp, inst, w.rows, w.depths, config=sliced)
        b = gpu_bounds(fsp, inst, w.rows, w.depths, config=whole)
        assert np.array_equal(a, b)
        assert np.array_equal(a[idx], oracle_bounds(w.p, w.rows[idx], w.depths[idx]))
        small = w.rows[:2000], w.depths[:2000]
        auto = fsp.fsp_tuned_config(inst, 2000)
        assert auto["kernel"] == fsp.FSP_KERNEL_LANES and auto["pairs_per_tile"] < 190
        assert np.array_equal(gpu_bounds(fsp, inst, *small), b[:2000])
    with fsp.Instance(w.p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        got = gpu_bounds(fsp, inst, w.rows[:3000], w.depths[:3000], config=sliced)
    want = oracle.Tables(w.p).lb_pool(w.rows[:3000], w.depths[:3000], threads=THREADS, release=oracle.RELEASE_EST)
    assert np.array_equal(got, want)
    p, rows, depths = pool(9, 45, 11, 1700, hi=20000)
    with fsp.Instance(p) as inst:
        assert inst.info().compact == 0
        got = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, warps_per_block=2, positions_per_tile=8,
                                                              staging=2, pairs_per_tile=32))
    assert np.array_equal(got, oracle_bounds(p, rows, depths))


@pytest.mark.parametrize("ts", [2, 3, 6])
@pytest.mark.parametrize("W,bps", [(1, 1), (2, 2)])
def test_tail_sliced_batches_match_oracle(gpu_lib, ts, W, bps):
    """Pools of more than one wave of block batches whose last partial wave
    is split by couples (tail_slices 2, 3 and 6 of the 6 groups at m = 20):
    the whole batches store their bounds, the tail's slices meet in the
    atomic max; the last batch is ragged and the pool holds invalid rows."""
    import torch
    fsp = gpu_lib
    slots = torch.cuda.get_device_properties(0).multi_processor_count * bps
    N = (slots + 37) * 32 * W + 19
    p, rows, depths = pool(640 + ts, 40, 20, N)
    depths[[5, N - 3]] = [-1, 41]
    rows[N - 1, :2] = [7, 7]
    depths[N - 1] = max(int(depths[N - 1]), 2)
    cfg = dict(kernel=2, staging=2, warps_per_block=W, blocks_per_sm=bps, positions_per_tile=12, tail_slices=ts)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
        whole = gpu_bounds(fsp, inst, rows, depths, config=dict(cfg, tail_slices=1))
    assert np.array_equal(got, whole)
    assert got[5] == got[N - 3] == got[N - 1] == fsp.FSP_LB_INVALID
    idx = np.concatenate([np.arange(0, N, 97), np.arange(N - 40 * 32 * W, N)])
    assert np.array_equal(got[idx], oracle_bounds(p, rows[idx], depths[idx]))


def test_couple_slices_refused_outside_streamed_and_split_staging(gpu_lib):
    import torch
    fsp = gpu_lib
    p, rows, depths = pool(2, 30, 12, 100)
    r, d = to_dev(rows, depths)
    with fsp.Instance(p) as inst:
        # slices throughout and slices of the last wave exclude each other
        with pytest.raises(fsp.FspError):
            fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=2, pairs_per_tile=32, tail_slices=2))
        for staging in (1, 3, 4):
            if staging != 3:  # split staging takes couple slices
                with pytest.raises(fsp.FspError):
                    fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=staging, pairs_per_tile=32))
            with pytest.raises(fsp.FspError):
                fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=staging, tail_slices=2))
            # all couples in one work item is every staging's own shape
            out = fsp.fsp_bound_pool(inst, r, d, config=dict(kernel=2, staging=staging, pairs_per_tile=66))
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), oracle_bounds(p, rows, depths))


def test_wide_records_match_oracle(gpu_lib):
    """Processing times above 255 select the 128-bit Johnson records."""
    fsp = gpu_lib
    p, rows, depths = pool(5, 60, 12, 2500, hi=20000)
    with fsp.Instance(p) as inst:
        assert inst.info().compact == 0
        got = gpu_bounds(fsp, inst, rows, depths)
        got_k1 = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=1, nodes_per_thread=1, blocks_per_sm=1,
                                                                   pairs_per_tile=5))
        got_lanes = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, warps_per_block=4,
                                                                      positions_per_tile=16, staging=2))
        got_res = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, warps_per_block=4, staging=1))
        got_split = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, warps_per_block=4,
                                                                      positions_per_tile=16, staging=3))
        got_warp = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, warps_per_block=4,
                                                                     positions_per_tile=8, staging=4))
    want = oracle_bounds(p, rows, depths)
    assert np.array_equal(got, want)
    assert np.array_equal(got_k1, want)
    assert np.array_equal(got_lanes, want)
    assert np.array_equal(got_res, want)
    assert np.array_equal(got_split, want)
    assert np.array_equal(got_warp, want)


def test_latencies_above_int16(gpu_lib):
    """Processing times up to 210,000 (128-bit records): minimum tails q_l
    far above 2^15, which the couple-lanes rows must hold in full.  On these
    pools about one node in twelve has a bound that a 16-bit q would change
    (checked on the CPU when the pools were chosen); every staging mode and
    the node-lockstep kernel must match the oracle."""
    fsp = gpu_lib
    rng = np.random.default_rng(41)
    for trial in range(8):
        n = int(rng.integers(3, 8))
        m = int(rng.integers(3, 10))
        p = rng.integers(1, 70000, (n, m)).astype(np.int32)
        p[:, 1] *= 3
        rows, depths = workloads.random_pool(rng, n, 300, max_depth=n)
        want = oracle_bounds(p, rows, depths)
        with fsp.Instance(p) as inst:
            assert inst.info().compact == 0
            cfgs = [None, dict(kernel=1, nodes_per_thread=2)]
            cfgs += [dict(kernel=2, warps_per_block=2, staging=st, positions_per_tile=0 if st == 1 else 4)
                     for st in (1, 2, 3, 4)]
            for cfg in cfgs:
                got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
                assert np.array_equal(got, want), (trial, cfg, np.nonzero(got != want)[0][:5])


def test_pair_tiled_500x20_matches_oracle(gpu_lib):
    """n=500, m=20: 190 couples x 500 entries do not fit in shared memory at
    once, so the tables are staged tile by tile."""
    fsp = gpu_lib
    w = workloads.named_pool("pool_500x20", N=1400)
    with fsp.Instance(w.p) as inst:
        got = gpu_bounds(fsp, inst, w.rows, w.depths)
    assert np.array_equal(got, oracle_bounds(w.p, w.rows, w.depths))


def test_maximum_sizes(gpu_lib):
    """n = 1024 jobs (the largest instance) and m = 32 machines."""
    fsp = gpu_lib
    for seed, n, m, N in ((11, 1024, 4, 300), (12, 30, 32, 400)):
        p, rows, depths = pool(seed, n, m, N)
        with fsp.Instance(p) as inst:
            got = gpu_bounds(fsp, inst, rows, depths)
            others = [gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, staging=st)) for st in (3, 4)]
        assert np.array_equal(got, oracle_bounds(p, rows, depths))
        for o in others:
            assert np.array_equal(o, got)


def test_edge_rows(gpu_lib):
    """depth 0, depth n (leaves: the bound is the makespan), equal times
    (every Johnson key ties), zero times, and invalid rows."""
    fsp = gpu_lib
    from oracle import brute
    n, m = 9, 4
    rng = np.random.default_rng(3)
    for p in (rng.integers(1, 100, (n, m), dtype=np.int32), np.full((n, m), 7, np.int32),
              np.zeros((n, m), np.int32), rng.integers(0, 2, (n, m), dtype=np.int32)):
        rows = np.tile(np.arange(n, dtype=np.int16), (12, 1))
        for i in range(12):
            rows[i] = rng.permutation(n)
        depths = np.array([0, n, n, 1, 3, n - 1, 0, 2, -1, n + 1, 4, 4], np.int32)
        rows[10, :4] = [0, 1, 1, 2]      # duplicate job
        rows[11, :4] = [0, 1, 9, 2]      # job out of range
        with fsp.Instance(p) as inst:
            got = gpu_bounds(fsp, inst, rows, depths)
            for staging in (2, 3, 4):
                cfg = dict(kernel=2, warps_per_block=2, positions_per_tile=4, staging=staging)
                assert np.array_equal(gpu_bounds(fsp, inst, rows, depths, config=cfg), got)
        want = oracle_bounds(p, rows, depths)
        assert np.array_equal(got, want)
        assert got[1] == brute.makespan(p, rows[1].tolist())
        assert got[8] == got[9] == got[10] == got[11] == fsp.FSP_LB_INVALID


def test_empty_and_single_pools(gpu_lib):
    import torch
    fsp = gpu_lib
    p, rows, depths = pool(1, 10, 5, 1)
    with fsp.Instance(p) as inst:
        assert gpu_bounds(fsp, inst, rows, depths).tolist() == oracle_bounds(p, rows, depths).tolist()
        e = torch.empty((0, 10), dtype=torch.int16, device="cuda")
        out = fsp.fsp_bound_pool(inst, e, torch.empty(0, dtype=torch.int32, device="cuda"))
        assert out.numel() == 0
        for staging in (3, 4):
            cfg = dict(kernel=2, warps_per_block=4, positions_per_tile=8, staging=staging)
            out = fsp.fsp_bound_pool(inst, e, torch.empty(0, dtype=torch.int32, device="cuda"), config=cfg)
            assert out.numel() == 0
            assert gpu_bounds(fsp, inst, rows, depths, config=cfg).tolist() == oracle_bounds(p, rows, depths).tolist()


def test_host_buffer_entry_point(gpu_lib):
    """fsp_bound_pool_host: pageable and pinned host buffers, several chunks."""
    import torch
    fsp = gpu_lib
    w = workloads.named_pool("pool_20x20", N=70001)
    want = oracle_bounds(w.p, w.rows, w.depths)
    with fsp.Instance(w.p) as inst:
        got = fsp.fsp_bound_pool_host(inst, w.rows, w.depths)
        assert np.array_equal(got, want)
        pr = torch.from_numpy(w.rows).pin_memory()
        pd = torch.from_numpy(w.depths).pin_memory()
        po = torch.empty(w.N, dtype=torch.int32).pin_memory()
        fsp.fsp_bound_pool_host(inst, pr, pd, po)
        assert np.array_equal(po.numpy(), want)


def test_host_entry_point_wave_chunks(gpu_lib):
    """Pools of two to nine waves of block batches: the host path stages
    them as a first chunk of two thirds of a wave and then whole waves (at
    most eight chunks, so the largest pool takes two waves per chunk); its
    bounds equal the device path's on every node and the oracle's on a
    sample, with and without a tuned shape."""
    import torch
    fsp = gpu_lib
    for N in (160001, 700001):
        w = workloads.named_pool("pool_20x20", N=N)
        r, d = to_dev(w.rows, w.depths)
        with fsp.Instance(w.p) as inst:
            dev = fsp.fsp_bound_pool(inst, r, d)
            torch.cuda.synchronize()
            dev = dev.cpu().numpy()
            assert np.array_equal(fsp.fsp_bound_pool_host(inst, w.rows, w.depths), dev)
            if N == 160001:
                fsp.fsp_autotune(inst, r, d)
                assert np.array_equal(fsp.fsp_bound_pool_host(inst, w.rows, w.depths), dev)
        idx = np.random.default_rng(N).choice(N, 3000, replace=False)
        assert np.array_equal(dev[idx], oracle_bounds(w.p, w.rows[idx], w.depths[idx]))


@pytest.mark.parametrize("n,m,N", [(20, 20, 1), (20, 20, 500), (30, 5, 40000), (64, 6, 9000)])
def test_host_entry_point_small_and_lockstep_pools(gpu_lib, n, m, N):
    """fsp_bound_pool_host on one-chunk pools, on a node-lockstep instance
    (m = 5: 10 couples, split 20/80) and on a depth-ordered one-chunk pool."""
    fsp = gpu_lib
    p, rows, depths = pool(7 * n + m, n, m, N)
    with fsp.Instance(p) as inst:
        got = fsp.fsp_bound_pool_host(inst, rows, depths)
    assert np.array_equal(got, oracle_bounds(p, rows, depths))


def test_side_stream_and_repeat_calls(gpu_lib):
    import torch
    fsp = gpu_lib
    p, rows, depths = pool(21, 30, 10, 4000)
    want = oracle_bounds(p, rows, depths)
    s = torch.cuda.Stream()
    with fsp.Instance(p) as inst:
        r, d = to_dev(rows, depths)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            outs = [fsp.fsp_bound_pool(inst, r, d, stream=s) for _ in range(3)]
        s.synchronize()
        for o in outs:
            assert np.array_equal(o.cpu().numpy(), want)


def test_full_size_20x20_pool(gpu_lib):
    """The 20x20 bounding pool (seed 1, 65,536 nodes), every node."""
    fsp = gpu_lib
    w = workloads.named_pool("pool_20x20")
    with fsp.Instance(w.p) as inst:
        got = gpu_bounds(fsp, inst, w.rows, w.depths)
    assert np.array_equal(got, oracle_bounds(w.p, w.rows, w.depths))


@pytest.mark.parametrize("name,sample", [("pool_200x20", 3000), ("pool_500x20", 600)])
def test_full_size_pools_sampled(gpu_lib, name, sample):
    """The 200x20 (262,144 nodes) and 500x20 (65,536 nodes) pools, bounded
    whole in the launch shape the benchmark uses; a seeded sample of nodes is
    recomputed by the oracle one by one."""
    fsp = gpu_lib
    w = workloads.named_pool(name)
    with fsp.Instance(w.p) as inst:
        got = gpu_bounds(fsp, inst, w.rows, w.depths)
        other = dict(kernel=fsp.FSP_KERNEL_LOCKSTEP)
        got_other = gpu_bounds(fsp, inst, w.rows, w.depths, config=other)
        for staging in (2, 3, 4):
            shape = dict(kernel=2, staging=staging, warps_per_block=8, blocks_per_sm=2,
                         positions_per_tile=8 if staging == 4 else 64)
            assert np.array_equal(gpu_bounds(fsp, inst, w.rows, w.depths, config=shape), got)
    assert np.array_equal(got, got_other)
    idx = np.sort(np.random.default_rng(123).choice(w.N, sample, replace=False))
    idx = np.unique(np.concatenate([idx, [0, w.N - 1]]))
    want = oracle_bounds(w.p, w.rows[idx], w.depths[idx])
    assert np.array_equal(got[idx], want)
    assert (got > 0).all()


def test_split_pool_larger_than_one_chunk(gpu_lib):
    """The split kernels bound pools above 2^20 nodes chunk by chunk through
    one scratch allocation: same bounds as the fused kernel, a sample checked
    against the oracle, the ragged last chunk included."""
    fsp = gpu_lib
    N = (1 << 20) + 4133
    p, rows, depths = pool(31, 12, 6, N)
    with fsp.Instance(p) as inst:
        split = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, staging=3, warps_per_block=6))
        fused = gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=2, staging=2, warps_per_block=6))
    assert np.array_equal(split, fused)
    idx = np.unique(np.concatenate([np.random.default_rng(5).choice(N, 4000, replace=False),
                                    np.arange((1 << 20) - 40, (1 << 20) + 40), [0, N - 1]]))
    assert np.array_equal(split[idx], oracle_bounds(p, rows[idx], depths[idx]))


def test_depth_ordered_pools_with_invalid_and_extreme_depths(gpu_lib):
    """Pools at and just above the size where the library bounds them in
    depth order (8,192 nodes, n >= 64 jobs), with invalid depths (-1, n + 1)
    and every depth from 0 to n mixed in; every bound lands at its node."""
    fsp = gpu_lib
    rng = np.random.default_rng(77)
    n, m = 64, 6
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    with fsp.Instance(p) as inst:
        for N in (8191, 8192, 8193, 20000):
            rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
            depths[rng.choice(N, 50, replace=False)] = -1
            depths[rng.choice(N, 50, replace=False)] = n + 1
            depths[:n + 1] = np.arange(n + 1)
            got = gpu_bounds(fsp, inst, rows, depths)
            assert np.array_equal(got, oracle_bounds(p, rows, depths)), N
            assert (got[(depths < 0) | (depths > n)] == fsp.FSP_LB_INVALID).all()


def test_depth_order_with_more_depth_bins_than_threads(gpu_lib):
    """Depth order of a pool whose jobs give more depth bins (n + 3 = 303)
    than the scatter kernel has threads, so each thread sums a segment of
    several bins: every bound lands at its node, invalid depths included."""
    fsp = gpu_lib
    rng = np.random.default_rng(78)
    n, m = 300, 4
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    with fsp.Instance(p) as inst:
        for N in (8192, 12345):
            rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
            depths[rng.choice(N, 40, replace=False)] = -1
            depths[rng.choice(N, 40, replace=False)] = n + 1
            depths[:n + 1] = np.arange(n + 1)
            got = gpu_bounds(fsp, inst, rows, depths)
            assert np.array_equal(got, oracle_bounds(p, rows, depths)), N


def test_host_entry_point_mixed_pinned_and_pageable(gpu_lib):
    """fsp_bound_pool_host with a mix of page-locked and pageable buffers
    (pinned rows, pageable depths) and with all three page-locked: both give
    the oracle's bounds."""
    import torch
    fsp = gpu_lib
    w = workloads.named_pool("pool_200x20", N=9000)
    want = oracle_bounds(w.p, w.rows, w.depths)
    with fsp.Instance(w.p) as inst:
        pr = torch.from_numpy(w.rows).pin_memory()
        po = torch.empty(w.N, dtype=torch.int32).pin_memory()
        fsp.fsp_bound_pool_host(inst, pr, w.depths, po)
        assert np.array_equal(po.numpy(), want)
        pd = torch.from_numpy(w.depths).pin_memory()
        po.zero_()
        fsp.fsp_bound_pool_host(inst, pr, pd, po)
        assert np.array_equal(po.numpy(), want)


@pytest.mark.parametrize("n,m", [(1, 2), (2, 2), (3, 2), (1, 5), (2, 7), (64, 2)])
def test_tiny_and_two_machine_instances(gpu_lib, n, m):
    """n = 1 and 2 jobs, m = 2 machines (one couple), every depth; at m = 2
    the root bound is Johnson's optimum (brute force over all orders)."""
    from oracle import brute
    fsp = gpu_lib
    p, rows, depths = pool(400 + 10 * n + m, n, m, 600)
    with fsp.Instance(p) as inst:
        got = gpu_bounds(fsp, inst, rows, depths)
        assert np.array_equal(got, oracle_bounds(p, rows, depths))
        if m == 2 and n <= 8:
            root = gpu_bounds(fsp, inst, np.zeros((1, n), np.int16), np.zeros(1, np.int32))
            assert root[0] == brute.optimum(p)[0]


def test_largest_processing_times(gpu_lib):
    """Processing times as large as the instance limit allows (sum of all
    p_jk just below 2^30): 128-bit records, every intermediate value near
    the int32 range."""
    fsp = gpu_lib
    rng = np.random.default_rng(9)
    n, m = 12, 6
    p = rng.integers(1, (2 ** 30 - 1) // (n * m), (n, m), dtype=np.int32)
    assert int(p.sum(dtype=np.int64)) < 2 ** 30
    rows, depths = workloads.random_pool(rng, n, 3000, max_depth=n + 1)
    with fsp.Instance(p) as inst:
        assert inst.info().compact == 0
        got = gpu_bounds(fsp, inst, rows, depths)
    assert np.array_equal(got, oracle_bounds(p, rows, depths))


def _every_path(fsp, inst, rows, depths):
    """Bounds of one pool from every kernel and staging mode that can take the
    instance, the batched launch and the allocation-free batched entry point."""
    import torch
    info = inst.info()
    cfgs = [None, dict(kernel=2, staging=2, warps_per_block=4, positions_per_tile=64),
            dict(kernel=2, staging=2, warps_per_block=8, pairs_per_tile=96),
            dict(kernel=2, staging=3, warps_per_block=4), dict(kernel=2, staging=4, warps_per_block=2),
            dict(kernel=1, nodes_per_thread=2)]
    if info.flags:
        cfgs.pop()  # per-job release times: couple-lanes kernels only
    if info.compact:  # global staging and two node sets per warp take two-word records only
        cfgs += [dict(kernel=2, staging=5, warps_per_block=4), dict(kernel=2, staging=5, warps_per_block=1,
                                                                    pairs_per_tile=32),
                 dict(kernel=2, staging=2, nodes_per_thread=56, warps_per_block=3, positions_per_tile=64),
                 dict(kernel=2, staging=2, nodes_per_thread=28, warps_per_block=5, positions_per_tile=32)]
    out = {str(c): gpu_bounds(fsp, inst, rows, depths, config=c) for c in cfgs}
    if info.compact:
        r, d = to_dev(rows, depths)
        o1 = torch.full((rows.shape[0],), -9, dtype=torch.int32, device="cuda")
        o2 = torch.full((rows.shape[0],), -9, dtype=torch.int32, device="cuda")
        with fsp.Batch([(inst, r, d, o1)]) as b:
            b.launch()
        fsp.fsp_bound_batch_noalloc([(inst, r, d, o2)])
        torch.cuda.synchronize()
        out["batch"] = o1.cpu().numpy()
        out["noalloc"] = o2.cpu().numpy()
    return out


@pytest.mark.parametrize("case", ["p200to255", "all255", "all255_per_job"])
def test_scaled_scan_exact_at_its_limits(gpu_lib, case):
    """The two-word records of compact instances hold 1024 s + j and
    1024 delta, and the couple-lanes scan keeps the slack scaled by 1024
    with a job in its low 10 bits.  The encoding is tightest where s and the
    job are both near their limits and the slack grows large: n = 1024 jobs
    (job bits up to 1023), m = 32 machines, times 200..255 (every s of the
    couple (0, 31) between 6,200 and 7,905; with m <= 32 and p <= 255, s
    never reaches 8,192), the last 34 jobs at 255 on machines 1..31, shallow
    prefixes so long scans run.  With all times 255 every Johnson order is a
    tie and every minimum tail is 31 x 255, the largest latency a compact
    record's int16 row holds.  Every kernel, staging mode and batched entry
    point must match the oracle bit for bit."""
    fsp = gpu_lib
    rng = np.random.default_rng(2024)
    n, m, N = 1024, 32, 160
    if case == "p200to255":
        p = rng.integers(200, 256, size=(n, m), dtype=np.int32)
        p[990:, 1:] = 255
    else:
        p = np.full((n, m), 255, np.int32)
    rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
    depths[: N // 2] = rng.integers(0, 64, N // 2)  # long scans
    depths[-3:] = [0, n - 1, n]
    per_job = case.endswith("per_job")
    with fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB if per_job else 0) as inst:
        assert inst.info().compact == 1
        got = _every_path(fsp, inst, rows, depths)
    want = oracle.Tables(p).lb_pool(rows, depths, threads=THREADS,
                                    release=oracle.RELEASE_EST if per_job else oracle.RELEASE_HEADS)
    for k, v in got.items():
        assert np.array_equal(v, want), (case, k, np.nonzero(v != want)[0][:5])


@pytest.mark.parametrize("top", [255, 256])
def test_compact_and_wide_records_at_the_switch(gpu_lib, top):
    """Largest processing time 255 keeps the compact two-word records, 256
    switches to 128-bit records (with m <= 32 a row sum s of 8,192 or more
    needs a time above 255, so the time decides); both sides of the switch
    must match the oracle on every path."""
    fsp = gpu_lib
    rng = np.random.default_rng(2025 + top)
    n, m, N = 300, 32, 400
    p = rng.integers(1, 256, size=(n, m), dtype=np.int32)
    p[n - 1, :] = 255
    p[n - 1, m - 1] = top
    rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
    with fsp.Instance(p) as inst:
        assert inst.info().compact == (1 if top == 255 else 0)
        got = _every_path(fsp, inst, rows, depths)
    want = oracle_bounds(p, rows, depths)
    for k, v in got.items():
        assert np.array_equal(v, want), (top, k, np.nonzero(v != want)[0][:5])
