"""fsp_branch_and_bound (GPU bounding) vs the oracle's DFS B&B and brute force:
same optimum, same node count (identical DFS semantics)."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_small_instance_optimum_and_node_count(gpu_lib):
    """8 jobs x 5 machines, seed 0, ub0 = max(quoted formula, identity
    makespan); checked against all 8! permutations."""
    fsp = gpu_lib
    p = workloads.small_bnb_instance()
    ub0 = max(workloads.trivial_ub(p), brute.makespan(p, range(8)))
    with fsp.Instance(p) as inst:
        st, best, perm, nodes = fsp.fsp_branch_and_bound(inst, ub0)
    ost, obest, operm, onodes = oracle.branch_and_bound(p, ub0)
    assert st == fsp.FSP_OK and ost == oracle.FO_OK
    assert best == obest == brute.optimum(p)[0] == 630
    assert nodes == onodes
    assert perm.tolist() == operm.tolist()
    assert brute.makespan(p, perm.tolist()) == best


@pytest.mark.parametrize("seed", range(8))
def test_random_instances(gpu_lib, seed):
    fsp = gpu_lib
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(2, 7))
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    ub0 = brute.makespan(p, range(n))
    with fsp.Instance(p) as inst:
        st, best, perm, nodes = fsp.fsp_branch_and_bound(inst, ub0)
    ost, obest, operm, onodes = oracle.branch_and_bound(p, ub0)
    assert (st, best, nodes) == (ost, obest, onodes)
    assert perm.tolist() == operm.tolist()


def test_not_found_below_optimum(gpu_lib):
    fsp = gpu_lib
    p = workloads.small_bnb_instance()
    with fsp.Instance(p) as inst:
        st, _, _, nodes = fsp.fsp_branch_and_bound(inst, 629)
    ost, _, _, onodes = oracle.branch_and_bound(p, 629)
    assert st == fsp.FSP_ENOTFOUND and ost == oracle.FO_ENOTFOUND and nodes == onodes


def test_twelve_job_search(gpu_lib):
    """A 12x5 search solved to optimality on both sides (same node count)."""
    fsp = gpu_lib
    p = np.random.default_rng(200).integers(1, 100, (12, 5), dtype=np.int32)
    ub0 = brute.makespan(p, range(12))
    with fsp.Instance(p) as inst:
        st, best, perm, nodes = fsp.fsp_branch_and_bound(inst, ub0)
    ost, obest, _, onodes = oracle.branch_and_bound(p, ub0)
    assert st == ost == fsp.FSP_OK and best == obest and nodes == onodes
    assert brute.makespan(p, perm.tolist()) == best


def test_iterated_greedy_upper_bound(gpu_lib):
    """The library's iterated greedy schedule is a permutation whose makespan
    (by the textbook recurrence) is the value returned, never above NEH's and
    never below the optimum: the brute-force optimum on 8-job instances, the
    oracle's stored optima on the 20-job serving searches."""
    import json
    import os
    fsp = gpu_lib
    rng = np.random.default_rng(77)
    for t in range(6):
        n, m = 8, int(rng.integers(2, 7))
        p = rng.integers(1, 100, (n, m), dtype=np.int32)
        opt, _ = brute.optimum(p)
        with fsp.Instance(p) as inst:
            neh_v, _ = fsp.fsp_neh(inst)
            v, perm = fsp.fsp_iterated_greedy(inst, iterations=200, seed=t)
            assert sorted(perm.tolist()) == list(range(n))
            assert v == brute.makespan(p, perm.tolist())
            assert opt <= v <= neh_v
            assert fsp.fsp_iterated_greedy(inst, iterations=200, seed=t)[0] == v  # deterministic
            assert fsp.fsp_iterated_greedy(inst, iterations=0, seed=t)[0] == neh_v
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "serving_optima.json")))["results"]
    probs = dict(workloads.serving_searches())
    for seed in (202, 209, 216, 218):
        with fsp.Instance(probs[seed]) as inst:
            v, perm = fsp.fsp_iterated_greedy(inst, iterations=1000, seed=1)
        assert v == brute.makespan(probs[seed], perm.tolist())
        assert golden[str(seed)]["opt"] is None or v >= golden[str(seed)]["opt"]
