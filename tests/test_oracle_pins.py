"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: every expected value comes
from a hand derivation (tests/golden/hand_3x3.json), from brute-force
enumeration over all orders (oracle/brute.py, which never uses Johnson's
rule), from a closed form, or from an invariant of the bound.
"""
import itertools
import json
import os
import random

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1208_3933_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_instance(rng, n, m, hi=99):
    return rng.integers(1, hi + 1, size=(n, m), dtype=np.int32)


def rand_prefix(rng, n, d):
    return [int(x) for x in rng.permutation(n)[:d]]


# ---------------------------------------------------------------- hand example
def test_hand_worked_3x3_tables_and_bounds():
    g = json.load(open(os.path.join(GOLDEN, "hand_3x3.json")))
    p = np.array(g["p"], np.int32)
    t = oracle.Tables(p)
    assert t.mm.tolist() == g["pairs"]
    assert t.lag.tolist() == g["lag"]
    assert t.jm.tolist() == g["jm"]
    for nd in g["nodes"]:
        lb, pairs = t.lb(nd["prefix"], return_pairs=True)
        assert pairs.tolist() == nd["pair_values"], nd
        assert lb == nd["lb"], nd
    for key, v in g["makespans"].items():
        assert brute.makespan(p, [int(x) for x in key.split(",")]) == v
    assert brute.optimum(p)[0] == g["optimum"]


# ------------------------------------------- per-couple value = brute minimum
@pytest.mark.parametrize("seed", range(12))
def test_pair_values_equal_enumerated_minimum(seed):
    """Johnson's rule with lags solves the relaxed two-machine problem of
    every couple exactly, so each couple's value must equal the minimum over
    all orders of the unscheduled jobs.  This pins JM, LM, RM, QM and the
    recurrence at once (a dropped lag, a wrong Johnson set or sort
    direction, a swapped M1/M2 or a wrong release or latency all break it)."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 7))
    m = int(rng.integers(2, 6))
    hi = [3, 9, 99][seed % 3]  # small ranges force many Johnson ties
    p = rand_instance(rng, n, m, hi)
    t = oracle.Tables(p)
    for _ in range(4):
        d = int(rng.integers(0, n))
        prefix = rand_prefix(rng, n, d)
        lb, pairs = t.lb(prefix, return_pairs=True)
        for c, (k, l) in enumerate(t.mm.tolist()):
            assert pairs[c] == brute.pair_minimum(p, prefix, k, l), (p.tolist(), prefix, k, l)
        assert lb == max(int(v) for v in pairs)


# -------------------------------------------------------------- closed form
def test_pair_values_match_max_plus_closed_form():
    """Second formula for one couple, over the filtered Johnson order
    j_1..j_u of the unscheduled jobs:
        t2 = max( r_l + sum_i b_i,  max_i ( r_k + sum_{i'<=i} a_i' + lag_i + sum_{i'>=i} b_i' ) )
    with a = p_jk, b = p_jl; the couple value is t2 + q_l."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        n = int(rng.integers(1, 12))
        m = int(rng.integers(2, 7))
        p = rand_instance(rng, n, m)
        t = oracle.Tables(p)
        prefix = rand_prefix(rng, n, int(rng.integers(0, n + 1)))
        r, q = brute.release_and_latency(p, prefix)
        _, pairs = t.lb(prefix, return_pairs=True)
        S = set(prefix)
        for c, (k, l) in enumerate(t.mm.tolist()):
            order = [int(j) for j in t.jm[c] if int(j) not in S]
            a = [int(p[j][k]) for j in order]
            b = [int(p[j][l]) for j in order]
            lag = [int(sum(p[j][k + 1:l])) for j in order]
            best = r[l] + sum(b)
            for i in range(len(order)):
                best = max(best, r[k] + sum(a[: i + 1]) + lag[i] + sum(b[i:]))
            assert pairs[c] == best + q[l]


# --------------------------------------------------------------- validity
@pytest.mark.parametrize("seed", range(8))
def test_lb_never_exceeds_best_completion(seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 8))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m)
    t = oracle.Tables(p)
    for d in range(0, n + 1):
        prefix = rand_prefix(rng, n, d)
        assert t.lb(prefix) <= brute.best_completion(p, prefix)


def test_lb_at_leaves_equals_makespan():
    rng = np.random.default_rng(3)
    for _ in range(50):
        n = int(rng.integers(1, 15))
        m = int(rng.integers(2, 9))
        p = rand_instance(rng, n, m)
        perm = rand_prefix(rng, n, n)
        assert oracle.Tables(p).lb(perm) == brute.makespan(p, perm)


def test_two_machines_root_bound_is_the_optimum():
    """m = 2: one couple, no lag, and Johnson's rule is exact (Section II-B)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        n = int(rng.integers(1, 8))
        p = rand_instance(rng, n, 2, hi=int(rng.choice([3, 99])))
        assert oracle.Tables(p).lb([]) == brute.optimum(p)[0]


def test_bound_is_monotone_along_branches():
    """LB(child) >= LB(parent): a child schedules one more job, which can only
    raise the release times and shrink the unscheduled set."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        n = int(rng.integers(2, 25))
        m = int(rng.integers(2, 8))
        p = rand_instance(rng, n, m, hi=int(rng.choice([5, 99])))
        t = oracle.Tables(p)
        perm = rand_prefix(rng, n, n)
        prev = t.lb([])
        for d in range(1, n + 1):
            cur = t.lb(perm[:d])
            assert cur >= prev
            prev = cur


def test_bound_does_not_depend_on_the_johnson_tie_break():
    """With times in 1..2 almost every job ties; the value still equals the
    enumerated minimum of every couple (checked above for random ties); here
    we relabel the jobs, which changes every index tie-break, and the bound
    of the same node must not move."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        n = int(rng.integers(2, 9))
        m = int(rng.integers(2, 6))
        p = rand_instance(rng, n, m, hi=2)
        relabel = rng.permutation(n)  # new index of old job j
        q = np.empty_like(p)
        q[relabel] = p
        prefix = rand_prefix(rng, n, int(rng.integers(0, n + 1)))
        assert oracle.Tables(p).lb(prefix) == oracle.Tables(q).lb([int(relabel[j]) for j in prefix])


def test_invalid_nodes_are_rejected():
    p = rand_instance(np.random.default_rng(8), 6, 3)
    t = oracle.Tables(p)
    assert t.lb([0, 0]) is None            # duplicate job
    assert t.lb([6]) is None               # job out of range
    assert t.lb([-1]) is None
    assert t.lb(list(range(7))) is None    # depth > n
    rows = np.zeros((3, 6), np.int16)
    rows[1, :2] = [3, 3]
    out = t.lb_pool(rows, np.array([-1, 2, 7], np.int32))
    assert out.tolist() == [-1, -1, -1]


# --------------------------------------------------------- branch and bound
def test_bnb_small_instance_matches_brute_force():
    """The plain-method instance (8 jobs x 5 machines, seed 0): the B&B
    optimum equals the optimum over all 8! permutations."""
    p = workloads.small_bnb_instance()
    opt, _ = brute.optimum(p)
    ub0 = max(workloads.trivial_ub(p), brute.makespan(p, range(8)))
    rc, best, perm, nodes = oracle.branch_and_bound(p, ub0)
    assert rc == oracle.FO_OK
    assert best == opt == 630
    assert brute.makespan(p, perm.tolist()) == best
    assert sorted(perm.tolist()) == list(range(8))
    assert nodes > 0


@pytest.mark.parametrize("seed", range(6))
def test_bnb_random_instances_match_brute_force(seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m)
    opt, _ = brute.optimum(p)
    ub0 = brute.makespan(p, range(n))
    rc, best, perm, _ = oracle.branch_and_bound(p, ub0)
    assert rc == oracle.FO_OK and best == opt
    assert brute.makespan(p, perm.tolist()) == opt


def test_bnb_reports_not_found_below_the_optimum():
    p = workloads.small_bnb_instance()
    rc, _, _, nodes = oracle.branch_and_bound(p, 629)
    assert rc == oracle.FO_ENOTFOUND and nodes >= 1
    rc, best, _, _ = oracle.branch_and_bound(p, 630)  # ub0 = opt is reachable
    assert rc == oracle.FO_OK and best == 630


def test_trivial_ub_formula_is_not_always_valid():
    """The quoted ub0 formula can fall below the optimum; the B&B must then
    report not-found rather than a wrong schedule."""
    p = np.array([[1, 10], [1, 10]], np.int32)
    assert workloads.trivial_ub(p) == 12 and brute.optimum(p)[0] == 21
    rc, _, _, _ = oracle.branch_and_bound(p, workloads.trivial_ub(p))
    assert rc == oracle.FO_ENOTFOUND


@pytest.mark.parametrize("release", [oracle.RELEASE_HEADS, oracle.RELEASE_EST])
@pytest.mark.parametrize("seed", range(4))
def test_bnb_subtree_optimum_is_the_best_completion(seed, release):
    """A search started at a prefix covers exactly the schedules that begin
    with it: its optimum is the brute-force best completion of the prefix
    (not-found when that exceeds ub0), and the smallest optimum over every
    prefix of one length is the brute-force optimum of the instance."""
    rng = np.random.default_rng(4200 + seed)
    n = int(rng.integers(3, 8))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m)
    opt, _ = brute.optimum(p)
    ub0 = opt + int(rng.integers(0, 40))
    for depth in (1, 2):
        found = []
        for prefix in itertools.permutations(range(n), depth):
            rc, best, perm, nodes = oracle.branch_and_bound(p, ub0, release, prefix)
            want = brute.best_completion(p, list(prefix))
            assert nodes >= 1
            if want <= ub0:
                assert rc == oracle.FO_OK and best == want, (prefix, best, want)
                assert perm.tolist()[:depth] == list(prefix)
                assert brute.makespan(p, perm.tolist()) == best
                found.append(best)
            else:
                assert rc == oracle.FO_ENOTFOUND, prefix
        assert min(found) == opt


@pytest.mark.parametrize("seed", range(6))
def test_bnb_with_per_job_release_matches_brute_force(seed):
    """The search bounded with the per-job release times reaches the
    brute-force optimum, and reports not-found one below it."""
    rng = np.random.default_rng(4300 + seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m)
    opt, _ = brute.optimum(p)
    rc, best, perm, _ = oracle.branch_and_bound(p, brute.makespan(p, range(n)), oracle.RELEASE_EST)
    assert rc == oracle.FO_OK and best == opt == brute.makespan(p, perm.tolist())
    rc, _, _, _ = oracle.branch_and_bound(p, opt - 1, oracle.RELEASE_EST)
    assert rc == oracle.FO_ENOTFOUND


def test_bnb_refuses_a_bad_prefix():
    p = workloads.small_bnb_instance()
    for bad in ((3, 3), (8,), (-1,)):
        with pytest.raises(ValueError):
            oracle.branch_and_bound(p, 1000, oracle.RELEASE_HEADS, bad)


# ----------------------------- the per-job reading of the release times (RM)
@pytest.mark.parametrize("seed", range(10))
def test_est_pair_values_equal_enumerated_minimum(seed):
    """With RM read as the earliest start of each unscheduled job on each
    machine, every couple's value is still the minimum over all orders of the
    relaxed two-machine problem, now released at min_j (C(prefix + [j], k) -
    p_jk) -- the start times found by appending each job to the prefix."""
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(2, 7))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m, [3, 9, 99][seed % 3])
    t = oracle.Tables(p)
    for _ in range(4):
        prefix = rand_prefix(rng, n, int(rng.integers(0, n + 1)))
        lb, pairs = t.lb(prefix, return_pairs=True, release=oracle.RELEASE_EST)
        for c, (k, l) in enumerate(t.mm.tolist()):
            assert pairs[c] == brute.pair_minimum(p, prefix, k, l, "est"), (p.tolist(), prefix, k, l)
        assert lb == max(int(v) for v in pairs)


@pytest.mark.parametrize("seed", range(8))
def test_est_bound_is_valid_and_at_least_the_default(seed):
    """The per-job release times are never earlier than the default ones, so
    the bound is at least the default bound, and it stays below the best
    completion of the node (a valid bound); at leaves it is the makespan."""
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(2, 8))
    m = int(rng.integers(2, 6))
    p = rand_instance(rng, n, m)
    t = oracle.Tables(p)
    for d in range(n + 1):
        prefix = rand_prefix(rng, n, d)
        est = t.lb(prefix, release=oracle.RELEASE_EST)
        assert t.lb(prefix) <= est <= brute.best_completion(p, prefix)
        if d == n:
            assert est == brute.makespan(p, prefix)


def test_est_pool_matches_single_nodes():
    rng = np.random.default_rng(4100)
    p = rand_instance(rng, 9, 6)
    rows, depths = workloads.random_pool(rng, 9, 300, max_depth=10)
    t = oracle.Tables(p)
    got = t.lb_pool(rows, depths, threads=3, release=oracle.RELEASE_EST)
    want = [t.lb(rows[i, :depths[i]].tolist(), release=oracle.RELEASE_EST) for i in range(300)]
    assert got.tolist() == [(-1 if w is None else w) for w in want]


# ------------------------------------------------- the pins catch mistakes
MUTANTS = {
    "dropped lag": ("for (int h = k + 1; h < l; ++h) lg += p[j * m + h];", ""),
    "set 2 ascending": ("items[j].key = -b;", "items[j].key = b;"),
    "set test reversed": ("if (p[j * m + k] <= p[j * m + l]) {", "if (p[j * m + k] >= p[j * m + l]) {"),
    "no latency": ("t2 += Q[M2];           /* latency of M2 */", ""),
    "release without heads": ("R[k] = C[k] > mh ? C[k] : mh;", "R[k] = C[k];"),
    "machines swapped in update": ("t2 += p[job * m + M2];", "t2 += p[job * m + M1];"),
    "scheduled jobs not filtered": ("if (sched[job]) continue; /* only unscheduled jobs */", ""),
    "est: machine availability ignored": ("est = C[k] > ready ? C[k] : ready;", "est = ready;"),
    "est: time of the wrong machine": ("int64_t ready = est + p[j * m + k - 1];", "int64_t ready = est + p[j * m + k];"),
    "est: largest start kept": ("if (R[k] < 0 || est < R[k]) R[k] = est;", "if (R[k] < 0 || est > R[k]) R[k] = est;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_detect_planted_mistakes(name, tmp_path):
    """Plants one plausible mistake in a copy of the oracle (on the CPU) and
    checks that the enumeration pins reject it."""
    import ctypes
    import subprocess

    src = open(os.path.join(os.path.dirname(oracle.__file__), "fsp_oracle.c")).read()
    old, new = MUTANTS[name]
    release = oracle.RELEASE_EST if name.startswith("est:") else oracle.RELEASE_HEADS
    assert src.count(old) == 1, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(mut)])
    lib = ctypes.CDLL(str(so))
    I32 = ctypes.POINTER(ctypes.c_int32)

    def mutant_lb(p, prefix):
        n, m = p.shape
        P = m * (m - 1) // 2
        mm = np.zeros((P, 2), np.int32); lag = np.zeros((P, n), np.int32); jm = np.zeros((P, n), np.int32)
        pc = np.ascontiguousarray(p, np.int32)
        lib.fo_tables(n, m, pc.ctypes.data_as(I32), mm.ctypes.data_as(I32), lag.ctypes.data_as(I32),
                      jm.ctypes.data_as(I32))
        row = np.zeros(n, np.int16); row[: len(prefix)] = prefix
        out = ctypes.c_int32(0)
        lib.fo_lb_ex(n, m, pc.ctypes.data_as(I32), mm.ctypes.data_as(I32), lag.ctypes.data_as(I32),
                     jm.ctypes.data_as(I32), row.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)),
                     len(prefix), release, None, ctypes.byref(out))
        return out.value

    rng = np.random.default_rng(99)
    caught = False
    for _ in range(60):
        n = int(rng.integers(2, 6)); m = int(rng.integers(2, 6))
        p = rand_instance(rng, n, m)
        prefix = rand_prefix(rng, n, int(rng.integers(0, n)))
        if mutant_lb(p, prefix) != brute.lb_by_enumeration(p, prefix, "est" if release else "heads"):
            caught = True
            break
    assert caught, f"mutant '{name}' survived the enumeration pin"


def test_neh_gives_a_valid_schedule_at_least_the_optimum():
    from oracle.neh import neh
    rng = np.random.default_rng(12)
    for _ in range(10):
        n = int(rng.integers(1, 8)); m = int(rng.integers(2, 5))
        p = rand_instance(rng, n, m)
        v, seq = neh(p)
        assert sorted(seq) == list(range(n))
        assert v == brute.makespan(p, seq) >= brute.optimum(p)[0]


def test_iterated_greedy_gives_a_valid_schedule_at_least_the_optimum():
    from oracle.ig import iterated_greedy
    from oracle.neh import neh
    rng = np.random.default_rng(13)
    for _ in range(8):
        n = int(rng.integers(1, 8)); m = int(rng.integers(2, 5))
        p = rand_instance(rng, n, m)
        v, seq = iterated_greedy(p, iterations=30, seed=1)
        assert sorted(seq) == list(range(n))
        assert v == brute.makespan(p, seq)
        assert brute.optimum(p)[0] <= v <= neh(p)[0]
