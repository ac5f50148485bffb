"""Per-job release times (fsp_instance_create_ex with
FSP_INSTANCE_RELEASE_PER_JOB): GPU bounds vs the oracle's RELEASE_EST
reading, element by element, for every couple-lanes staging mode; the bound
is never below the default one; the B&B reaches the same optimum."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def pool(seed, n, m, N):
    rng = np.random.default_rng(seed)
    p = rng.integers(1, 100, size=(n, m), dtype=np.int32)
    rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
    return p, rows, depths


def gpu_bounds(fsp, inst, rows, depths, config=None):
    import torch
    r = torch.from_numpy(np.ascontiguousarray(rows)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(depths)).cuda()
    out = fsp.fsp_bound_pool(inst, r, d, config=config)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("staging,positions", [(0, 0), (1, 0), (2, 8), (3, 8), (4, 8)])
@pytest.mark.parametrize("nm", [(17, 5), (40, 20), (70, 12), (33, 27)])
def test_per_job_release_matches_oracle(gpu_lib, staging, positions, nm):
    fsp = gpu_lib
    n, m = nm
    p, rows, depths = pool(7 + n, n, m, 1500)
    want = oracle.Tables(p).lb_pool(rows, depths, threads=8, release=oracle.RELEASE_EST)
    cfg = None if staging == 0 else dict(kernel=2, warps_per_block=4, positions_per_tile=positions, staging=staging)
    with fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        assert inst.info().flags == fsp.FSP_INSTANCE_RELEASE_PER_JOB
        got = gpu_bounds(fsp, inst, rows, depths, config=cfg)
    assert np.array_equal(got, want)


def test_per_job_release_is_at_least_the_default(gpu_lib):
    fsp = gpu_lib
    w = workloads.named_pool("pool_200x20", N=20000)
    with fsp.Instance(w.p) as plain, fsp.Instance(w.p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as per_job:
        a = gpu_bounds(fsp, plain, w.rows, w.depths)
        b = gpu_bounds(fsp, per_job, w.rows, w.depths)
    assert (b >= a).all() and (b > a).any()
    idx = np.random.default_rng(3).choice(w.N, 400, replace=False)
    assert np.array_equal(b[idx], oracle.Tables(w.p).lb_pool(w.rows[idx], w.depths[idx], threads=8,
                                                                release=oracle.RELEASE_EST))


def test_per_job_release_edge_rows_and_lockstep_refused(gpu_lib):
    fsp = gpu_lib
    n, m = 9, 4
    rng = np.random.default_rng(5)
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    rows = np.stack([rng.permutation(n) for _ in range(8)]).astype(np.int16)
    depths = np.array([0, n, n - 1, 1, -1, n + 1, 4, 3], np.int32)
    rows[6, :4] = [0, 1, 1, 2]
    with fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        got = gpu_bounds(fsp, inst, rows, depths)
        with pytest.raises(fsp.FspError) as e:
            gpu_bounds(fsp, inst, rows, depths, config=dict(kernel=fsp.FSP_KERNEL_LOCKSTEP))
        assert e.value.status == fsp.FSP_EINVAL
    want = oracle.Tables(p).lb_pool(rows, depths, release=oracle.RELEASE_EST)
    assert np.array_equal(got, want)
    assert got[1] == brute.makespan(p, rows[1].tolist())
    assert got[4] == got[5] == got[6] == fsp.FSP_LB_INVALID


def test_per_job_release_in_batches_and_searches(gpu_lib):
    """Mixed batch of default and per-job instances; B&B optimum with the
    tighter bound (host-driven and device-driven searches)."""
    import torch
    fsp = gpu_lib
    specs = [(20, 5, 3000, 0), (50, 10, 2000, 1), (20, 20, 1000, 1), (30, 12, 777, 0)]
    pools, want = [], []
    for i, (n, m, N, fl) in enumerate(specs):
        p, rows, depths = pool(60 + i, n, m, N)
        inst = fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB if fl else 0)
        r = torch.from_numpy(rows).cuda(); d = torch.from_numpy(depths).cuda()
        pools.append((inst, r, d, torch.empty(N, dtype=torch.int32, device="cuda")))
        want.append(oracle.Tables(p).lb_pool(rows, depths, threads=8, release=fl))
    with fsp.Batch(pools) as b:
        b.launch()
        torch.cuda.synchronize()
    for (inst, _, _, out), wv in zip(pools, want):
        assert np.array_equal(out.cpu().numpy(), wv)
        inst.close()
    p = workloads.small_bnb_instance()
    ub0 = max(workloads.trivial_ub(p), brute.makespan(p, range(8)))
    with fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB) as inst:
        st, best, perm, nodes = fsp.fsp_branch_and_bound(inst, ub0)
        st2, best2, _, nodes2 = fsp.fsp_branch_and_bound_device(inst, ub0, expand=8)
    assert st == st2 == fsp.FSP_OK and best == best2 == 630
    assert brute.makespan(p, perm.tolist()) == 630
