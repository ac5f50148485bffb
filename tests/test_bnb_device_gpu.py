"""fsp_branch_and_bound_device (branching, bounding and elimination on the
device) vs brute force and the oracle's DFS B&B: same optimum, a valid
optimal permutation, the not-found and node-limit outcomes."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.neh import neh
from oracle import brute
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "serving_optima.json")


@pytest.mark.parametrize("expand", [1, 3, 256])
def test_small_instance(gpu_lib, expand):
    """8 jobs x 5 machines, seed 0: optimum 630 (all 8! permutations)."""
    fsp = gpu_lib
    p = workloads.small_bnb_instance()
    ub0 = max(workloads.trivial_ub(p), brute.makespan(p, range(8)))
    with fsp.Instance(p) as inst:
        st, best, perm, nodes = fsp.fsp_branch_and_bound_device(inst, ub0, expand=expand)
    assert st == fsp.FSP_OK
    assert best == brute.optimum(p)[0] == 630
    assert sorted(perm.tolist()) == list(range(8))
    assert brute.makespan(p, perm.tolist()) == best
    assert nodes >= 1


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("expand", [1, 64])
def test_random_instances(gpu_lib, seed, expand):
    """n in 1..8, m in 2..6: optimum = brute force; n = 1 has a single leaf."""
    fsp = gpu_lib
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(2, 7))
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    ub0 = brute.makespan(p, range(n))
    with fsp.Instance(p) as inst:
        st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, ub0, expand=expand)
    assert st == fsp.FSP_OK
    assert best == brute.optimum(p)[0]
    assert brute.makespan(p, perm.tolist()) == best


def test_not_found_below_optimum(gpu_lib):
    fsp = gpu_lib
    p = workloads.small_bnb_instance()
    with fsp.Instance(p) as inst:
        st, _, _, nodes = fsp.fsp_branch_and_bound_device(inst, 629, expand=16)
    assert st == fsp.FSP_ENOTFOUND and nodes >= 1


def test_node_limit(gpu_lib):
    fsp = gpu_lib
    p = np.random.default_rng(200).integers(1, 100, (12, 5), dtype=np.int32)
    with fsp.Instance(p) as inst:
        st, _, _, nodes = fsp.fsp_branch_and_bound_device(inst, 10 ** 6, expand=4, node_limit=50)
    assert st == fsp.FSP_ETIMEDOUT and nodes >= 50


def test_twelve_job_search(gpu_lib):
    """12 x 5: the device search and the oracle's search reach the same optimum."""
    fsp = gpu_lib
    p = np.random.default_rng(200).integers(1, 100, (12, 5), dtype=np.int32)
    ub0 = brute.makespan(p, range(12))
    ost, obest, _, _ = oracle.branch_and_bound(p, ub0)
    assert ost == oracle.FO_OK
    with fsp.Instance(p) as inst:
        for expand in (1, 32, 1024):
            st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, ub0, expand=expand)
            assert st == fsp.FSP_OK and best == obest
            assert brute.makespan(p, perm.tolist()) == best


@pytest.mark.parametrize("seed", [200, 201, 203])
def test_serving_searches_reach_the_stored_optimum(gpu_lib, seed):
    """20-job searches of the serving workload, from the oracle's NEH upper
    bound, against the optima the oracle stored in tests/golden."""
    fsp = gpu_lib
    rec = json.load(open(GOLDEN))["results"][str(seed)]
    p = dict(workloads.serving_searches())[seed]
    with fsp.Instance(p) as inst:
        st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, neh(p)[0], expand=256)
    assert st == fsp.FSP_OK and best == rec["opt"]
    assert brute.makespan(p, perm.tolist()) == best


@pytest.mark.parametrize("expand", [1, 5, 128])
def test_best_first_reaches_the_optimum(gpu_lib, expand):
    """Best-first selection (the k open nodes of smallest bound per round):
    same optimum as brute force / the oracle, on small and 12-job instances."""
    fsp = gpu_lib
    p = workloads.small_bnb_instance()
    ub0 = max(workloads.trivial_ub(p), brute.makespan(p, range(8)))
    with fsp.Instance(p) as inst:
        st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, ub0, expand=expand,
                                                            selection=fsp.FSP_SELECT_BEST_FIRST)
    assert st == fsp.FSP_OK and best == 630 and brute.makespan(p, perm.tolist()) == 630
    p = np.random.default_rng(200).integers(1, 100, (12, 5), dtype=np.int32)
    ub0 = brute.makespan(p, range(12))
    _, obest, _, _ = oracle.branch_and_bound(p, ub0)
    with fsp.Instance(p) as inst:
        st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, ub0, expand=expand,
                                                            selection=fsp.FSP_SELECT_BEST_FIRST)
    assert st == fsp.FSP_OK and best == obest and brute.makespan(p, perm.tolist()) == best


@pytest.mark.parametrize("seed", range(6))
def test_best_first_random_instances(gpu_lib, seed):
    fsp = gpu_lib
    rng = np.random.default_rng(950 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(2, 7))
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    with fsp.Instance(p) as inst:
        st, best, perm, _ = fsp.fsp_branch_and_bound_device(inst, brute.makespan(p, range(n)), expand=3,
                                                            selection=fsp.FSP_SELECT_BEST_FIRST)
        st2, _, _, _ = fsp.fsp_branch_and_bound_device(inst, brute.optimum(p)[0] - 1, expand=3,
                                                       selection=fsp.FSP_SELECT_BEST_FIRST)
    assert st == fsp.FSP_OK and best == brute.optimum(p)[0]
    assert st2 == fsp.FSP_ENOTFOUND


@pytest.mark.parametrize("seed", [200, 202])
def test_best_first_is_deterministic(gpu_lib, seed):
    """The best-first selection takes ties by stack position (no atomic
    order decides), so a search expands the same nodes on every run: same
    node count and the same optimal permutation, twice, at the optimum the
    oracle stored."""
    fsp = gpu_lib
    rec = json.load(open(GOLDEN))["results"][str(seed)]
    p = dict(workloads.serving_searches([seed]))[seed]
    runs = []
    with fsp.Instance(p) as inst:
        for _ in range(2):
            st, best, perm, nodes = fsp.fsp_branch_and_bound_device(inst, neh(p)[0], expand=256,
                                                                    selection=fsp.FSP_SELECT_BEST_FIRST)
            assert st == fsp.FSP_OK and best == rec["opt"]
            assert brute.makespan(p, perm.tolist()) == best
            runs.append((nodes, perm.tolist()))
    assert runs[0] == runs[1]
