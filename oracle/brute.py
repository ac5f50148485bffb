"""Brute-force enumerations that pin the oracle (tiny instances only).

TEST INFRASTRUCTURE ONLY.  Pure Python, written from the definitions of the
permutation flow-shop (Section II-B of Melab et al.) and of the relaxed
two-machine problem with lags that the bound of Section II-C solves.  Nothing
here uses Johnson's rule: every minimum is taken over all orders, so a wrong
Johnson order, lag, release time or latency in the oracle shows up as a
mismatch.
"""
from __future__ import annotations

import itertools


def completion_times(p, seq, m=None):
    """C(seq, k) for every machine k: each job visits M_1..M_m in order, each
    machine serves the jobs in the order of ``seq`` one at a time."""
    if m is None:
        m = len(p[0])
    C = [0] * m
    for j in seq:
        prev = 0
        for k in range(m):
            C[k] = max(C[k], prev) + int(p[j][k])
            prev = C[k]
    return C


def makespan(p, seq):
    """C_max of a complete permutation (completion on the last machine)."""
    return completion_times(p, seq)[-1]


def best_completion(p, prefix):
    """Minimum makespan over every completion of ``prefix`` (n' ! orders)."""
    n = len(p)
    rest = [j for j in range(n) if j not in set(prefix)]
    return min(makespan(p, list(prefix) + list(o)) for o in itertools.permutations(rest))


def optimum(p):
    """Optimal makespan over all n! permutations, and one optimal order."""
    n = len(p)
    best, arg = None, None
    for o in itertools.permutations(range(n)):
        v = makespan(p, o)
        if best is None or v < best:
            best, arg = v, o
    return best, list(arg)


def release_and_latency(p, prefix):
    """r_k = max(C(prefix,k), min over unscheduled j of sum_{h<k} p_jh) and
    q_l = min over unscheduled j of sum_{h>l} p_jh (0 when none is left)."""
    n, m = len(p), len(p[0])
    U = [j for j in range(n) if j not in set(prefix)]
    C = completion_times(p, prefix, m)
    r, q = [], []
    for k in range(m):
        if U:
            head = min(sum(int(p[j][h]) for h in range(k)) for j in U)
            tail = min(sum(int(p[j][h]) for h in range(k + 1, m)) for j in U)
        else:
            head, tail = 0, 0
        r.append(max(C[k], head))
        q.append(tail)
    return r, q


def release_by_appending(p, prefix):
    """The per-job reading of the release times: r_k = min over unscheduled j
    of the time job j would start on machine k if it were scheduled right
    after the prefix, C(prefix + [j], k) - p_jk; r_k = C(prefix, k) when no
    job is left.  Written from the flow-shop recurrence, not from a formula
    for earliest starts."""
    n, m = len(p), len(p[0])
    U = [j for j in range(n) if j not in set(prefix)]
    if not U:
        return completion_times(p, prefix, m)
    r = []
    for k in range(m):
        r.append(min(completion_times(p, list(prefix) + [j], m)[k] - int(p[j][k]) for j in U))
    return r


def two_machine_value(p, order, k, l, rk, rl, ql):
    """The relaxed problem on couple (M_k, M_l): machines between k and l
    become a lag (sum of the job's times strictly between them); machine k is
    free at rk, machine l at rl; the last job still needs ql after M_l."""
    t1, t2 = rk, rl
    for j in order:
        lag = sum(int(p[j][h]) for h in range(k + 1, l))
        t1 = t1 + int(p[j][k])
        t2 = max(t2, t1 + lag) + int(p[j][l])
    return t2 + ql


def pair_minimum(p, prefix, k, l, release="heads"):
    """Minimum of two_machine_value over every order of the unscheduled jobs;
    release = "heads" (the default reading) or "est" (release_by_appending)."""
    n = len(p)
    r, q = release_and_latency(p, prefix)
    if release == "est":
        r = release_by_appending(p, prefix)
    U = [j for j in range(n) if j not in set(prefix)]
    return min(two_machine_value(p, o, k, l, r[k], r[l], q[l]) for o in itertools.permutations(U))


def lb_by_enumeration(p, prefix, release="heads"):
    """max over couples k<l of pair_minimum: the bound computed with no
    Johnson order at all."""
    m = len(p[0])
    return max(pair_minimum(p, prefix, k, l, release) for k in range(m) for l in range(k + 1, m))
