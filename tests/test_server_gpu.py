"""The continuous-batching bounding server: every request's bounds equal the
same pool bounded alone (bit-exact), under concurrency, admission by device
budget, cancellation, shutdown; and served DFS searches reach the oracle's
optimum."""
import threading

import numpy as np
import pytest

import oracle
from oracle.neh import neh
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def make_pools(fsp, specs, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n, m, N in specs:
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
        out.append((fsp.Instance(p), rows, depths))
    return out


def alone(fsp, inst, rows, depths):
    import torch
    r = torch.from_numpy(rows).cuda()
    d = torch.from_numpy(depths).cuda()
    o = fsp.fsp_bound_pool(inst, r, d)
    torch.cuda.synchronize()
    return o.cpu().numpy()


def test_each_result_is_the_same_alone_and_in_the_mix(gpu_lib):
    fsp = gpu_lib
    specs = [(20, 5, 700), (50, 10, 3000), (200, 20, 2500), (20, 20, 33), (100, 12, 1500), (7, 3, 1)]
    pools = make_pools(fsp, specs, 1)
    ref = [alone(fsp, *p) for p in pools]
    for (inst, rows, depths), r in zip(pools, ref):  # the alone results are the oracle's
        assert np.array_equal(r, oracle.Tables(inst.p).lb_pool(rows, depths, threads=16))
    with fsp.Server(hbm_budget_bytes=64 << 20, slots=3) as srv:
        errors = []

        def client(cid):
            rng = np.random.default_rng(100 + cid)
            for _ in range(12):
                k = int(rng.integers(0, len(pools)))
                inst, rows, depths = pools[k]
                req = srv.submit(inst, rows, depths)
                st = req.wait(60_000_000)
                if st != fsp.FSP_OK or not np.array_equal(req.out, ref[k]):
                    errors.append((cid, k, st))
                req.release()

        threads = [threading.Thread(target=client, args=(c,)) for c in range(8)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(120)
        assert not errors, errors[:5]
        st = srv.stats()
        assert st["pools_done"] == 8 * 12
        assert st["batches"] <= st["pools_done"]
        assert st["p99_us"] >= st["p50_us"] > 0
    for inst, _, _ in pools:
        inst.close()


def test_admission_by_budget(gpu_lib):
    """A pool larger than the whole arena is refused at once; pools that fit
    only one at a time are admitted in turn and all complete exactly."""
    fsp = gpu_lib
    (inst, rows, depths), = make_pools(fsp, [(200, 20, 6000)], 2)
    per_pool = 6000 * 200 * 2 + 2 * 6000 * 4
    with fsp.Server(hbm_budget_bytes=per_pool // 2) as small:
        with pytest.raises(fsp.FspError) as e:
            small.submit(inst, rows, depths)
        assert e.value.status == fsp.FSP_EBUSY
    want = alone(fsp, inst, rows, depths)
    with fsp.Server(hbm_budget_bytes=int(per_pool * 1.5)) as one_at_a_time:
        reqs = [one_at_a_time.submit(inst, rows, depths) for _ in range(4)]
        for r in reqs:
            assert r.wait(60_000_000) == fsp.FSP_OK
            assert np.array_equal(r.out, want)
        assert one_at_a_time.stats()["batches"] == 4
    inst.close()


def test_cancel_timeout_and_shutdown(gpu_lib):
    fsp = gpu_lib
    (inst, rows, depths), = make_pools(fsp, [(200, 20, 40000)], 3)
    per_pool = 40000 * 200 * 2 + 2 * 40000 * 4
    want = alone(fsp, inst, rows, depths)
    with fsp.Server(hbm_budget_bytes=int(per_pool * 1.2)) as srv:
        a = srv.submit(inst, rows, depths)
        b = srv.submit(inst, rows, depths)  # waits for a's memory
        c = b.cancel()
        if c == fsp.FSP_OK:
            assert b.wait(0) == fsp.FSP_EBUSY
        else:  # b was admitted already and runs to completion
            assert c == fsp.FSP_EBUSY and b.wait(60_000_000) == fsp.FSP_OK and np.array_equal(b.out, want)
        assert a.wait(60_000_000) == fsp.FSP_OK and np.array_equal(a.out, want)
        srv.shutdown()
        with pytest.raises(fsp.FspError) as e:
            srv.submit(inst, rows, depths)
        assert e.value.status == fsp.FSP_EBUSY
    with fsp.Server() as srv:
        big = srv.submit(inst, rows, depths)
        st = big.wait(0)
        assert st in (fsp.FSP_ETIMEDOUT, fsp.FSP_OK)
        assert big.wait(60_000_000) == fsp.FSP_OK and np.array_equal(big.out, want)
    inst.close()


@pytest.mark.parametrize("seed", [200, 203, 205, 206, 211, 213])
def test_served_search_reaches_the_oracle_optimum(gpu_lib, seed):
    """20-job searches of the serving loop (m=5), with the oracle's optimum
    as ub0 so both sides explore small trees."""
    fsp = gpu_lib
    p = dict(workloads.serving_searches())[seed]
    ost, opt, _, _ = oracle.branch_and_bound(p, neh(p)[0])
    assert ost == oracle.FO_OK
    from oracle import brute
    with fsp.Instance(p) as inst, fsp.Server() as srv:
        for expand in (1, 16, 256):
            st, best, perm, nodes = srv.search(inst, opt, expand=expand)
            assert st == fsp.FSP_OK and best == opt, (expand, best, opt)
            assert brute.makespan(p, perm.tolist()) == opt
            assert sorted(perm.tolist()) == list(range(20))
        st, _, _, _ = srv.search(inst, opt - 1, expand=64)
        assert st == fsp.FSP_ENOTFOUND


def test_concurrent_served_searches(gpu_lib):
    """Eight searches at once share one server; every optimum is right."""
    fsp = gpu_lib
    seeds = [200, 203, 205, 206, 211, 213, 201, 208]
    probs = dict(workloads.serving_searches())
    opts = {s: oracle.branch_and_bound(probs[s], neh(probs[s])[0])[1] for s in seeds}
    insts = {s: fsp.Instance(probs[s]) for s in seeds}
    results = {}
    with fsp.Server(slots=2) as srv:
        def run(s):
            results[s] = srv.search(insts[s], opts[s], expand=32)

        threads = [threading.Thread(target=run, args=(s,)) for s in seeds]
        for t in threads:
            t.start()
        for t in threads:
            t.join(300)
        for s in seeds:
            st, best, _, _ = results[s]
            assert st == fsp.FSP_OK and best == opts[s], s
        assert srv.stats()["mean_pools_per_batch"] >= 1.0
    for inst in insts.values():
        inst.close()


@pytest.mark.parametrize("searchers", [1, 3, 8])
def test_cooperating_searchers_reach_the_optimum(gpu_lib, searchers):
    """fsp_server_solve: several searchers with one shared incumbent and work
    stealing reach the optimum the oracle stored (20x5 serving searches, NEH
    start) and brute force on the 8x5 instance; below the optimum nothing is
    found; a node limit cuts the search."""
    import json
    import os
    fsp = gpu_lib
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "serving_optima.json")))["results"]
    probs = dict(workloads.serving_searches())
    from oracle import brute
    with fsp.Server() as srv:
        for seed in (200, 201, 203):
            rec = golden[str(seed)]
            with fsp.Instance(probs[seed]) as inst:
                st, best, perm, nodes, _ = srv.solve(inst, neh(probs[seed])[0], searchers=searchers, expand=32)
                assert st == fsp.FSP_OK and best == rec["opt"], (seed, best, rec["opt"])
                assert brute.makespan(probs[seed], perm.tolist()) == best
                assert nodes >= 1
        p = workloads.small_bnb_instance()
        with fsp.Instance(p) as inst:
            st, best, perm, _, _ = srv.solve(inst, 10 ** 6, searchers=searchers, expand=4)
            assert st == fsp.FSP_OK and best == 630 == brute.makespan(p, perm.tolist())
            st, _, _, _, _ = srv.solve(inst, 629, searchers=searchers, expand=4)
            assert st == fsp.FSP_ENOTFOUND
            st, _, _, nodes, _ = srv.solve(inst, 10 ** 6, searchers=searchers, expand=1, node_limit=20)
            assert st in (fsp.FSP_ETIMEDOUT, fsp.FSP_OK) and nodes >= 1


def test_server_with_per_job_release_instances(gpu_lib):
    """Pools of instances created with per-job release times go through the
    server's batched launches with the same bounds as alone."""
    fsp = gpu_lib
    rng = np.random.default_rng(31)
    insts = []
    for n, m, N in [(30, 10, 2000), (60, 20, 1500)]:
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
        insts.append((fsp.Instance(p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB), p, rows, depths))
    with fsp.Server(slots=2) as srv:
        for inst, p, rows, depths in insts:
            req = srv.submit(inst, rows, depths)
            assert req.wait(60_000_000) == fsp.FSP_OK
            want = oracle.Tables(p).lb_pool(rows, depths, threads=8, release=oracle.RELEASE_EST)
            assert np.array_equal(req.out, want)
            assert np.array_equal(req.out, alone(fsp, inst, rows, depths))
            req.release()
    for inst, _, _, _ in insts:
        inst.close()


def test_page_locked_pools_are_bounded_in_place(gpu_lib):
    """Requests whose rows, depths and bounds all live in page-locked host
    memory are bounded in place (no copy, no arena space) and batched with
    staged requests of pageable memory; every result equals the oracle's.
    A server whose arena holds none of the page-locked pools still serves
    them."""
    import torch
    fsp = gpu_lib
    specs = [(20, 10, 900), (200, 20, 1200), (20, 5, 40), (60, 20, 700), (7, 3, 1)]
    pools = make_pools(fsp, specs, 9)
    pinned = []
    for inst, rows, depths in pools:
        r = torch.from_numpy(rows).pin_memory().numpy()
        d = torch.from_numpy(depths).pin_memory().numpy()
        o = torch.full((depths.shape[0],), -5, dtype=torch.int32).pin_memory().numpy()
        pinned.append((inst, r, d, o))
    want = [oracle.Tables(inst.p).lb_pool(rows, depths, threads=16) for inst, rows, depths in pools]
    with fsp.Server(hbm_budget_bytes=64 << 10, slots=2) as srv:
        for rep in range(3):
            reqs = [srv.submit(inst, r, d, out=o) for inst, r, d, o in pinned]
            small = [srv.submit(inst, rows[:5], depths[:5]) for inst, rows, depths in pools]
            for q, (_, _, _, o), w in zip(reqs, pinned, want):
                assert q.wait(60_000_000) == fsp.FSP_OK
                assert np.array_equal(o, w)
                q.release()
            for q, w in zip(small, want):
                assert q.wait(60_000_000) == fsp.FSP_OK
                assert np.array_equal(q.out, w[:5])
                q.release()
            for _, _, _, o in pinned:
                o.fill(-5)
        assert srv.stats()["arena_bytes_used"] == 0
    for inst, _, _ in pools:
        inst.close()


@pytest.mark.parametrize("seed,m", [(200, 5), (203, 5), (210, 5)])
def test_plain_search_is_the_served_search(gpu_lib, seed, m):
    """fsp_server_search without a server bounds every pool by its own plain
    launch: the same search, so the same optimum, node count and schedule
    as through the server, and the optimum the oracle stored."""
    import json
    import os
    fsp = gpu_lib
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "serving_optima.json")))["results"]
    p = dict(workloads.serving_searches())[seed]
    assert p.shape[1] == m
    from oracle import brute
    with fsp.Instance(p) as inst, fsp.Server() as srv:
        ub0, _ = fsp.fsp_iterated_greedy(inst, iterations=500, seed=3)
        served = srv.search(inst, ub0, expand=64)
        plain = fsp.fsp_search_plain(inst, ub0, expand=64)
    assert served[0] == plain[0] and served[1] == plain[1] and served[3] == plain[3]
    assert np.array_equal(served[2], plain[2])
    opt = served[1] if served[0] == fsp.FSP_OK else ub0  # not found below ub0: ub0 is optimal
    assert opt == golden[str(seed)]["opt"]
    if served[0] == fsp.FSP_OK:
        assert brute.makespan(p, served[2].tolist()) == opt
